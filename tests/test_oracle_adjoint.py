"""Pin for oracle/adjoint.py: the adjoint gradient of a pressure misfit with
respect to per-cell log K equals central finite differences."""

import numpy as np

from oracle import E0, paper_element
from oracle.adjoint import gradient_logK, solve_u_p
from synth import fields, hex_mesh, prism_mesh
from synth.voronoi import voronoi_mesh


def _check(mesh, spec, seed, flux_term=False):
    """flux_term: the misfit also weighs the flux DOFs (w . u, w random),
    which exercises the flux part of the adjoint right-hand side and its
    sign relative to the pressure part (the system is solved for -p)."""
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(mesh.n_cells)
    prob = fields.sine_problem()
    u0, p0 = solve_u_p(mesh, spec, theta, prob.f, prob.gD)
    ptarget = rng.standard_normal(p0.size) * 0.1
    w = None

    def loss(u, p):
        val = 0.5 * np.sum((p - ptarget) ** 2)
        return val + (w @ u if flux_term else 0.0)

    def dL(u, p):
        return (w.copy() if flux_term else np.zeros_like(u)), p - ptarget

    w = rng.standard_normal(u0.size) * 0.05

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


def test_adjoint_flux_and_pressure_misfit():
    _check(prism_mesh(2), paper_element(1), 3, flux_term=True)
    _check(voronoi_mesh(25, seed=6, lloyd=2), E0, 4, flux_term=True)


def test_adjoint_K2_hex():
    """The paper's k = 2 element (four pressure moments per cell): the same
    contraction with the cell's k = 2 mass matrix."""
    _check(hex_mesh(2), paper_element(2), 5, flux_term=True)
