"""vem_residual_norm_noalloc: the residual norm for callers that cannot let a
library allocate device memory (their device memory belongs to a framework
allocator with its own pool or budget, or they cannot afford the device-wide
synchronisation of cudaFree).

The entry point is checked through the C-ABI against the residual that the
existing vem_solve entry point reports, on two calls in a row, and against
NumPy on a matrix of many 2048-row tiles with a partial last tile.  This file
is named so that pytest collects it last."""

import numpy as np
import pytest

from synth import fields, hex_mesh, prism_mesh


def _system(vs, mesh, seed):
    """A stopped iterate of a K1 solve (residual far from rounding level), the
    assembled matrix and right-hand side, and vem_solve's statistics."""
    rng = np.random.default_rng(seed)
    K = fields.K_lognormal(mesh.n_cells, seed=seed + 1, sigma=1.0)
    s = vs.Solver(mesh, element=vs.VEM_ELEMENT_K1, krylov=vs.VEM_KRYLOV_FGMRES,
                  precond=vs.VEM_PREC_BLOCK_TRI, maxit=4, rtol=1e-14, inner_rtol=1e-6)
    s.set_coefficient(K)
    s.set_source(rng.standard_normal(mesh.n_cells), None)
    u, p, st = s.solve(allow_not_converged=True)
    A, rhs = s.system()
    s.close()
    assert st["relres"] > 1e-6
    return A, rhs, np.concatenate([u, -p]), st


def _call_twice(vs, A, rhs, xh):
    import torch
    dev = "cuda"
    rp = torch.from_numpy(A.indptr.astype(np.int64)).to(dev)
    col = torch.from_numpy(A.indices.astype(np.int32)).to(dev)
    val = torch.from_numpy(A.data).to(dev)
    x = torch.from_numpy(xh).to(dev)
    b = torch.from_numpy(rhs).to(dev)
    out = []
    for _ in range(2):
        o = torch.full((3,), float("nan"), dtype=torch.float64, device=dev)
        vs.residual_norm_noalloc(rp, col, val, x, b, o, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        out.append(o.cpu().numpy())
    return out


@pytest.fixture(scope="module")
def built():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    return vemsolve


@pytest.fixture(scope="module")
def vs(built):
    import torch
    assert torch.cuda.is_available()
    return built


@pytest.mark.gpu
def test_residual_norm_noalloc_matches_vem_solve(vs):
    A, rhs, x, st = _system(vs, prism_mesh(4), 12)
    out = _call_twice(vs, A, rhs, x)
    for o in out:
        assert o[2] == pytest.approx(st["relres"], rel=1e-12)
        assert o[1] == pytest.approx(np.linalg.norm(rhs), rel=1e-12)
        assert o[0] == pytest.approx(np.linalg.norm(rhs - A @ x), rel=1e-9)
    assert np.array_equal(out[0], out[1])


@pytest.mark.gpu
def test_residual_norm_noalloc_many_tiles(vs):
    """12^3 hexahedra, K1: 23,760 rows = 11 full 2048-row tiles and a partial
    one, so the per-tile partial sums and their combination over many tiles
    run; both outputs and their ratio against NumPy and vem_solve."""
    A, rhs, x, st = _system(vs, hex_mesh(12), 21)
    assert A.shape[0] % 2048 != 0 and A.shape[0] > 4 * 2048
    out = _call_twice(vs, A, rhs, x)
    r = np.linalg.norm(rhs - A @ x)
    for o in out:
        assert o[0] == pytest.approx(r, rel=1e-9)
        assert o[1] == pytest.approx(np.linalg.norm(rhs), rel=1e-12)
        assert o[2] == pytest.approx(st["relres"], rel=1e-12)
    assert np.array_equal(out[0], out[1])


def test_residual_norm_noalloc_rejects_oversize(built):
    """More rows than the static scratch covers: refused before any GPU work."""
    import ctypes
    vs = built
    dummy = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    st = vs.lib().vem_residual_norm_noalloc(2048 * 65536 + 1, dummy, dummy, dummy, dummy, dummy, dummy, None)
    assert st == 1


def test_residual_norm_noalloc_binding_refuses_host_arrays():
    """The binding passes raw device pointers, so host (NumPy) arrays and
    wrong dtypes are refused before the library is called."""
    import torch

    from paper_1901_02330_gb300 import vemsolve as vs
    rp = np.array([0, 1], dtype=np.int64)
    with pytest.raises(TypeError):
        vs.residual_norm_noalloc(rp, np.zeros(1, np.int32), np.zeros(1), np.zeros(1), np.zeros(1), np.zeros(3))
    t = torch.zeros(1, dtype=torch.float64)
    with pytest.raises((TypeError, ValueError)):
        vs.residual_norm_noalloc(torch.tensor([0, 1]), torch.zeros(1, dtype=torch.int32), t, t, t,
                                 torch.zeros(3, dtype=torch.float64))
