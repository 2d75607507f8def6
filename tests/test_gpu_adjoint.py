"""Adjoint gradients d loss / d log K through the C-ABI (vem_adjoint) and the
torch.autograd binding: against the oracle's adjoint gradient and against
central finite differences of the GPU forward solve."""

import numpy as np
import pytest

from oracle import E0, paper_element
from oracle.adjoint import gradient_logK
from synth import fields, prism_mesh
from synth.voronoi import voronoi_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    return vemsolve


CASES = {"E0-cvt": (lambda: voronoi_mesh(60, seed=5, lloyd=3), E0, 0),
         "K1-prism": (lambda: prism_mesh(3), paper_element(1), 1)}


@pytest.mark.parametrize("flux_term", [False, True], ids=["p-misfit", "u-and-p-misfit"])
@pytest.mark.parametrize("case", list(CASES))
def test_adjoint_matches_oracle(vs, case, flux_term):
    """flux_term: the loss also has a term w . u on the flux DOFs, so dL/du
    enters the adjoint right-hand side next to dL/dp."""
    mk, spec, elem = CASES[case]
    mesh = mk()
    rng = np.random.default_rng(7)
    theta = rng.standard_normal(mesh.n_cells)
    ptarget = 0.1 * rng.standard_normal(mesh.n_cells)
    prob = fields.sine_problem()
    s = vs.Solver(mesh, element=elem, krylov=1, precond=1, rtol=1e-13, inner_rtol=1e-13)
    s.set_coefficient(np.exp(theta))
    s.set_data(prob.f, prob.gD)
    u, p, st = s.solve()
    w = 0.05 * rng.standard_normal(u.size) if flux_term else np.zeros(u.size)
    g, ast = s.adjoint(w if flux_term else None, p - ptarget)
    u_o, p_o, g_o = gradient_logK(mesh, spec, theta, prob.f, prob.gD,
                                  lambda u_, p_: (w.copy(), p_ - ptarget))
    assert np.linalg.norm(g - g_o) <= 1e-8 * np.linalg.norm(g_o)
    s.close()


def test_autograd_against_finite_differences(vs):
    import torch
    from paper_1901_02330_gb300.autograd import solve
    mesh = voronoi_mesh(80, seed=2, lloyd=4)
    rng = np.random.default_rng(3)
    prob = fields.sine_problem()
    s = vs.Solver(mesh, element=0, krylov=1, precond=1, rtol=1e-13, inner_rtol=1e-13, device_io=1,
                  stream=torch.cuda.current_stream().cuda_stream)
    s.set_data(prob.f, prob.gD)
    theta = torch.tensor(rng.standard_normal(mesh.n_cells), device="cuda", requires_grad=True)
    ptarget = torch.tensor(0.1 * rng.standard_normal(mesh.n_cells), device="cuda")

    def loss_of(th):
        u, p = solve(th, s)
        return 0.5 * torch.sum((p - ptarget) ** 2)

    L = loss_of(theta)
    L.backward()
    g = theta.grad.detach().cpu().numpy()
    eps = 1e-6
    with torch.no_grad():
        for P in rng.choice(mesh.n_cells, size=8, replace=False):
            tp = theta.detach().clone()
            tm = theta.detach().clone()
            tp[P] += eps
            tm[P] -= eps
            fd = (loss_of(tp).item() - loss_of(tm).item()) / (2 * eps)
            assert abs(fd - g[P]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (P, fd, g[P])
    s.close()


def test_adjoint_needs_a_solve(vs):
    s = vs.Solver(prism_mesh(2))
    with pytest.raises(vs.VemError) as e:
        s.adjoint(None, np.ones(s.n_cells))
    assert e.value.code == 1
