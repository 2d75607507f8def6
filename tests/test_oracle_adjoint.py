"""Pin for oracle/adjoint.py: the adjoint gradient of a pressure misfit with
respect to per-cell log K equals central finite differences."""

import numpy as np

from oracle import E0, paper_element
from oracle.adjoint import gradient_logK, solve_u_p
from synth import fields, prism_mesh
from synth.voronoi import voronoi_mesh


def _check(mesh, spec, seed):
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(mesh.n_cells)
    prob = fields.sine_problem()
    ptarget = rng.standard_normal(mesh.n_cells) * 0.1

    def loss(u, p):
        return 0.5 * np.sum((p - ptarget) ** 2)

    def dL(u, p):
        return np.zeros_like(u), p - ptarget

    u, p, g = gradient_logK(mesh, spec, theta, prob.f, prob.gD, dL)
    eps = 1e-6
    for P in rng.choice(mesh.n_cells, size=5, replace=False):
        tp, tm = theta.copy(), theta.copy()
        tp[P] += eps
        tm[P] -= eps
        fd = (loss(*solve_u_p(mesh, spec, tp, prob.f, prob.gD)) -
              loss(*solve_u_p(mesh, spec, tm, prob.f, prob.gD))) / (2 * eps)
        assert abs(fd - g[P]) <= 1e-6 * max(abs(fd), 1e-3 * np.abs(g).max()), (P, fd, g[P])


def test_adjoint_E0_voronoi():
    _check(voronoi_mesh(30, seed=5, lloyd=2), E0, 1)


def test_adjoint_K1_prism():
    _check(prism_mesh(2), paper_element(1), 2)
