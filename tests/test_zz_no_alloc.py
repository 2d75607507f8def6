"""vem_residual_norm_noalloc: the residual norm for callers that cannot let a
library allocate device memory (their device memory belongs to a framework
allocator with its own pool or budget, or they cannot afford the device-wide
synchronisation of cudaFree).

The entry point is checked through the C-ABI against the residual that the
existing vem_solve entry point reports, on two calls in a row.  This file is
named so that pytest collects it last."""

import numpy as np
import pytest

from synth import fields, prism_mesh

pytestmark = pytest.mark.gpu


def test_residual_norm_noalloc_matches_vem_solve():
    import torch

    from paper_1901_02330_gb300 import build, vemsolve as vs
    build.build()
    assert torch.cuda.is_available()
    mesh = prism_mesh(4)
    rng = np.random.default_rng(12)
    K = fields.K_lognormal(mesh.n_cells, seed=13, sigma=1.0)
    s = vs.Solver(mesh, element=vs.VEM_ELEMENT_K1, krylov=vs.VEM_KRYLOV_FGMRES,
                  precond=vs.VEM_PREC_BLOCK_TRI, maxit=4, rtol=1e-14, inner_rtol=1e-6)
    s.set_coefficient(K)
    s.set_source(rng.standard_normal(mesh.n_cells), None)
    # a stopped iterate, so the residual is far from rounding level
    u, p, st = s.solve(allow_not_converged=True)
    A, rhs = s.system()
    s.close()
    assert st["relres"] > 1e-6

    dev = "cuda"
    rp = torch.from_numpy(A.indptr.astype(np.int64)).to(dev)
    col = torch.from_numpy(A.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(A.data).to(dev)
    x = torch.from_numpy(np.concatenate([u, -p])).to(dev)
    b = torch.from_numpy(rhs).to(dev)
    out = []
    for _ in range(2):
        o = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
        vs.residual_norm_noalloc(rp, col, val, x, b, o, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        out.append(o.cpu().numpy())
    for o in out:
        assert o[2] == pytest.approx(st["relres"], rel=1e-12)
        assert o[1] == pytest.approx(np.linalg.norm(rhs), rel=1e-12)
        assert o[0] == pytest.approx(np.linalg.norm(rhs - A @ np.concatenate([u, -p])), rel=1e-9)
    assert np.array_equal(out[0], out[1])


def test_residual_norm_noalloc_rejects_oversize():
    """More rows than the static scratch covers: refused before any GPU work."""
    import ctypes

    from paper_1901_02330_gb300 import vemsolve as vs
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    st = vs.lib().vem_residual_norm_noalloc(2048 * 65536 + 1, dummy, dummy, dummy, dummy, dummy, dummy, None)
    assert st == 1
