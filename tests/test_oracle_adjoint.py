"""Pin for oracle/adjoint.py: the adjoint gradient of a pressure misfit with
respect to per-cell log K equals central finite differences."""

import numpy as np

from oracle import E0, paper_element
from oracle.adjoint import gradient_logK, solve_u_p
from synth import fields, hex_mesh, prism_mesh
from synth.voronoi import voronoi_mesh


def _check(mesh, spec, seed, flux_term=False, eps=1e-6):
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
    contraction with the cell's k = 2 mass matrix.  Its direct solves carry
    ~1e-14 relative rounding in the loss, ~1e-8 in a difference quotient of
    step 1e-6 against gradient entries of ~1e-2, so the step is 1e-5 here
    (truncation ~1e-10)."""
    _check(hex_mesh(2), paper_element(2), 5, flux_term=True, eps=1e-5)


def _complex_step_check(mesh, spec, seed):
    """Complex-step derivative (Squire & Trapp, SIAM Rev. 40 (1998)): with
    theta_P -> theta_P + i h, nu_P = exp(-theta_P) becomes nu_P exp(-i h),
    so M -> M + (exp(-i h) - 1) M_P with M_P the cell's scaled local matrix;
    dL/dtheta_P = Im L(theta + i h e_P) / h to rounding for the analytic
    misfit L = 1/2 sum (p - p_target)^2 (no conjugation).  No step-size
    trade-off, so every cell's entry is checked at 1e-9 relative, small
    ones included."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla

    from oracle import assemble
    rng = np.random.default_rng(seed)
    theta = rng.standard_normal(mesh.n_cells)
    prob = fields.sine_problem()
    nu = np.exp(-theta)
    sys_ = assemble(mesh, spec, nu, f=prob.f, gD=prob.gD, keep_local=True)
    ptarget = 0.1 * rng.standard_normal(sys_.n_p)
    _, _, g = gradient_logK(mesh, spec, theta, prob.f, prob.gD, lambda u, p: (np.zeros_like(u), p - ptarget))
    A = sys_.saddle().tocsc().astype(np.complex128)
    b = sys_.rhs().astype(np.complex128)
    h = 1e-30
    n = sys_.n
    for P in range(mesh.n_cells):
        dm = sys_.dofmap[P]
        MP = sys_.local[P]["M"]
        dA = sp.csr_matrix(((np.expm1(-1j * h) * MP).ravel(), (np.repeat(dm, dm.size), np.tile(dm, dm.size))),
                           shape=(n, n))
        x = spla.spsolve((A + dA).tocsc(), b)
        p = -x[sys_.n_u:]
        L = 0.5 * np.sum((p - ptarget) ** 2)
        d = L.imag / h
        assert abs(d - g[P]) <= 1e-9 * abs(d) + 1e-14 * np.abs(g).max(), (P, d, g[P])


def test_adjoint_complex_step_E0_voronoi():
    _complex_step_check(voronoi_mesh(20, seed=8, lloyd=2), E0, 6)


def test_adjoint_complex_step_K1_prism():
    _complex_step_check(prism_mesh(2), paper_element(1), 7)


def test_krylov_option_matches_direct():
    """gradient_logK(solver='krylov') (FGMRES to 1e-14 with the exact-S block
    preconditioner) agrees with the direct factorisation."""
    mesh = voronoi_mesh(200, seed=9, lloyd=3)
    rng = np.random.default_rng(8)
    theta = rng.standard_normal(mesh.n_cells)
    pt = 0.1 * rng.standard_normal(mesh.n_cells)
    prob = fields.sine_problem()

    def dL(u, p):
        return np.zeros_like(u), p - pt
    _, _, gd = gradient_logK(mesh, E0, theta, prob.f, prob.gD, dL)
    _, _, gk = gradient_logK(mesh, E0, theta, prob.f, prob.gD, dL, solver="krylov")
    assert np.abs(gk - gd).max() <= 1e-12 * np.abs(gd).max()
