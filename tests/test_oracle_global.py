"""Pins for oracle/assemble.py, solvers.py and errors.py: patch tests,
conservation, convergence rates, the Schur complement on cubes, Krylov
solvers against the direct solve and against SciPy."""

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import E0, assemble, element, errors, paper_element, solvers
from oracle.element import interpolate
from oracle.monomials import eval_mono3, mono3
from synth import affine, fields, hex_mesh, octa_mesh, prism_mesh, tet_mesh
from synth.voronoi import voronoi_mesh

A_SHEAR = np.array([[1.0, 0.3, 0.1], [0.0, 0.8, -0.2], [0.1, 0.0, 1.2]])
MESHES = {
    "hex": lambda: hex_mesh(3),
    "tet": lambda: tet_mesh(2),
    "prism": lambda: prism_mesh(2),
    "sheared": lambda: affine(hex_mesh(2), A_SHEAR, (0.1, 0.0, -0.3)),
    "octa": lambda: octa_mesh(2),
    "voronoi": lambda: voronoi_mesh(30, seed=3, lloyd=0),
    "cvt": lambda: voronoi_mesh(40, seed=3, lloyd=5),
}


def _interp_all(sys, spec, v):
    uI = np.zeros(sys.n_u)
    for c, cell in enumerate(sys.cells):
        uI[sys.dofmap[c]] = interpolate(cell, spec, v)
    return uI


@pytest.mark.parametrize("mesh", list(MESHES))
@pytest.mark.parametrize("spec,probname", [(E0, "linear"), (paper_element(1), "linear"),
                                           (paper_element(1), "quadratic")],
                         ids=["E0-lin", "E1-lin", "E1-quad"])
def test_patch(mesh, spec, probname):
    """Constant K: if p in P_{kp+1} (flux in [P_kp]^3) the discrete solution is
    the DOF interpolant of the exact flux and the cell moments of p."""
    m = MESHES[mesh]()
    K = 2.5
    prob = fields.linear_problem(K=K) if probname == "linear" else fields.quadratic_problem(K=K)
    sys = assemble(m, spec, np.full(m.n_cells, 1.0 / K), f=prob.f, gD=prob.gD, keep_local=True)
    u, p = solvers.solve_direct(sys)
    uI = _interp_all(sys, spec, prob.u)
    pI = np.array([(cell.qw @ prob.p(cell.qp)) / cell.volume for cell in sys.cells])
    np.testing.assert_allclose(u, uI, atol=1e-11 * max(1, np.abs(uI).max()))
    np.testing.assert_allclose(p, pI, atol=1e-11)


def _quadratic_and_cubic(K):
    """p in P_2 and p in P_3 with constant K: u = -K grad p, f = div u."""
    def p2(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return 0.7 * X * X - X * Y + 0.3 * Z * Z + 0.5 * Y * Z - 0.2 * X + Y

    def u2(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return -K * np.stack([1.4 * X - Y - 0.2, -X + 0.5 * Z + 1.0, 0.6 * Z + 0.5 * Y], 1)

    def f2(x):
        return np.full(x.shape[0], -K * 2.0)

    def p3(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return X ** 3 - 2 * X * Y * Y + 0.5 * Z ** 3 + X * Y * Z + Y * Y - 0.4 * Z

    def u3(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return -K * np.stack([3 * X * X - 2 * Y * Y + Y * Z, -4 * X * Y + X * Z + 2 * Y,
                              1.5 * Z * Z + X * Y - 0.4], 1)

    def f3(x):
        X, Z = x[:, 0], x[:, 2]
        return -K * (2 * X + 2 + 3 * Z)

    return {"quadratic": (p2, u2, f2), "cubic": (p3, u3, f3)}


def _p1_moments(cells, q):
    """Pressure DOFs of the k = 2 element: (1/|P|) int_P q m_a, m_a the scaled
    P_1 monomials of the cell (eq. presMom)."""
    return np.concatenate([(cell.qw * q(cell.qp)) @ eval_mono3(mono3(1), cell.qp, cell.centroid, cell.diameter)
                           / cell.volume for cell in cells])


def _exact_face_rule(F, rule=None):
    """The face's own integration rule (exact to degree 8) in place of the
    degree-4 boundary data rule."""
    return F.qp, F.qw


@pytest.mark.parametrize("mesh", ["tet", "prism", "voronoi"])
def test_patch_k2_dirichlet_radon_rule(mesh):
    """With Radon's degree-5 fan rule for the Dirichlet term the cubic k = 2
    patch holds on triangular and Voronoi faces as well."""
    spec = paper_element(2)
    m = MESHES[mesh]()
    K = 1.7
    p_ex, u_ex, f_ex = _quadratic_and_cubic(K)["cubic"]
    sys = assemble(m, spec, np.full(m.n_cells, 1.0 / K), f=f_ex, gD=p_ex, keep_local=True, bface_rule="radon5")
    u, p = solvers.solve_direct(sys)
    uI = _interp_all(sys, spec, u_ex)
    np.testing.assert_allclose(u, uI, atol=1e-10 * np.abs(uI).max())
    np.testing.assert_allclose(p, _p1_moments(sys.cells, p_ex), atol=1e-10 * np.abs(p).max())


@pytest.mark.parametrize("mesh", list(MESHES))
@pytest.mark.parametrize("probname", ["quadratic", "cubic"])
def test_patch_k2_dirichlet(mesh, probname):
    """k = 2 with pressure data on the whole boundary, constant K: for p in
    P_3 (flux in [P_2]^3) u_h is the interpolant of the exact flux and p_h the
    P_1 moments of p.  The boundary term -int_f g_D m^f needs degree
    deg(p) + 2 = 5, which the default boundary rule of k = 2 (Radon's
    degree 5, boundary_rule) integrates exactly on every face shape."""
    spec = paper_element(2)
    m = MESHES[mesh]()
    K = 1.7
    p_ex, u_ex, f_ex = _quadratic_and_cubic(K)[probname]
    sys = assemble(m, spec, np.full(m.n_cells, 1.0 / K), f=f_ex, gD=p_ex, keep_local=True)
    assert sys.n_p == 4 * m.n_cells and not sys.multiplier
    u, p = solvers.solve_direct(sys)
    uI = _interp_all(sys, spec, u_ex)
    pI = _p1_moments(sys.cells, p_ex)
    np.testing.assert_allclose(u, uI, atol=1e-10 * max(1, np.abs(uI).max()))
    np.testing.assert_allclose(p, pI, atol=1e-10 * max(1, np.abs(pI).max()))


def test_k2_cubic_patch_needs_an_exact_boundary_rule(monkeypatch):
    """Why k = 2 takes a degree-5 boundary rule: Dunavant's degree-4 rule
    misses the degree-5 part of g_D m^f for a cubic g_D on triangular faces,
    so the cubic k = 2 patch is not reproduced there; an exact face rule
    changes g alone (M, B and F are the same matrices) and restores it."""
    spec = paper_element(2)
    assert element.boundary_rule(spec) == "radon5" and element.boundary_rule(paper_element(1)) == "dunavant4"
    m = tet_mesh(2)
    K = 1.7
    p_ex, u_ex, f_ex = _quadratic_and_cubic(K)["cubic"]
    sys = assemble(m, spec, np.full(m.n_cells, 1.0 / K), f=f_ex, gD=p_ex, keep_local=True, bface_rule="dunavant4")
    u, _ = solvers.solve_direct(sys)
    uI = _interp_all(sys, spec, u_ex)
    assert np.abs(u - uI).max() > 1e-6 * np.abs(uI).max()
    monkeypatch.setattr(element, "load_face_points", _exact_face_rule)
    ex = assemble(m, spec, np.full(m.n_cells, 1.0 / K), f=f_ex, gD=p_ex)
    assert abs(ex.M - sys.M).max() == 0.0 and abs(ex.B - sys.B).max() == 0.0
    np.testing.assert_array_equal(ex.F, sys.F)
    assert np.abs(ex.g - sys.g).max() > 1e-6 * np.abs(ex.g).max()
    ue, _ = solvers.solve_direct(ex)
    np.testing.assert_allclose(ue, uI, atol=1e-10 * np.abs(uI).max())


@pytest.mark.parametrize("spec", [E0, paper_element(1), paper_element(2)], ids=lambda s: s.name)
def test_local_conservation(spec):
    """B u_h = F: div u_h equals the projection of f on every cell."""
    m = prism_mesh(2)
    nu = fields.K_lognormal(m.n_cells, seed=4)
    sys = assemble(m, spec, nu, f=fields.sine_problem().f, gD=fields.sine_problem().gD)
    u, p = solvers.solve_direct(sys)
    np.testing.assert_allclose(sys.B @ u, sys.F, atol=1e-12 * np.abs(sys.F).max())


@pytest.mark.slow
@pytest.mark.parametrize("spec,rv,rq", [(E0, 1.0, 1.0), (paper_element(1), 2.0, 1.0),
                                        (paper_element(2), 3.0, 2.0)], ids=["E0", "E1", "E2"])
def test_convergence_rates(spec, rv, rq):
    """Sine solution on 4^3 -> 8^3 cubes: observed slopes of e_v, e_q against
    h (eq. meshSize) at least the expected rates - 0.2.  Expected: pressure
    O(h^k) (P_{k-1} pressure), flux O(h^{k+1}) for the paper's k = 1, 2 and
    O(h) for E0 -- Remark 4.1 prints the two rates the other way round; a
    P_{k-1} pressure cannot converge faster than O(h^k) in L2."""
    prob = fields.sine_problem()
    hs, ev, eq = [], [], []
    for n in (4, 8):
        m = hex_mesh(n)
        nu = np.ones(m.n_cells)
        sys = assemble(m, spec, nu, f=prob.f, gD=prob.gD, keep_local=True)
        u, p = solvers.solve_direct(sys)
        a, b = errors.indicators(sys, sys.cells, sys.dofmap, u, p, prob.u, prob.p, nu)
        hs.append(errors.mesh_size(sys.cells))
        ev.append(a)
        eq.append(b)
    sv = np.log(ev[1] / ev[0]) / np.log(hs[1] / hs[0])
    sq = np.log(eq[1] / eq[0]) / np.log(hs[1] / hs[0])
    assert sv >= rv - 0.2 and sq >= rq - 0.2, (sv, sq)
    assert hs[0] == pytest.approx(np.sqrt(3) / 4)


def test_schur_on_uniform_cubes():
    """E0 on cubes of side a: S = B diag(M)^{-1} B^T couples neighbours with
    -(4a/3)/(nu_P + nu_Q); a Dirichlet face adds (4a/3)/nu_P to the diagonal
    (diag(M) on a face is (3/4) a^3 times the sum of its cells' nu)."""
    n = 3
    a = 1.0 / n
    m = hex_mesh(n)
    nu = fields.K_lognormal(m.n_cells, seed=9, sigma=1.0)
    sys = assemble(m, E0, nu)
    S = solvers.schur(sys).toarray()
    ref = np.zeros_like(S)
    idx = lambda i, j, k: (i * n + j) * n + k
    for i in range(n):
        for j in range(n):
            for k in range(n):
                P = idx(i, j, k)
                for d in range(3):
                    for s in (-1, 1):
                        q = [i, j, k]
                        q[d] += s
                        if 0 <= q[d] < n:
                            Q = idx(*q)
                            w = (4 * a / 3) / (nu[P] + nu[Q])
                            ref[P, Q] -= w
                            ref[P, P] += w
                        else:
                            ref[P, P] += (4 * a / 3) / nu[P]
    np.testing.assert_allclose(S, ref, rtol=1e-12, atol=1e-14)


@pytest.fixture(scope="module")
def small_system():
    m = prism_mesh(2)
    nu = fields.K_lognormal(m.n_cells, seed=11)
    sys = assemble(m, paper_element(1), nu, f=fields.sine_problem().f, gD=fields.linear_problem().gD)
    return sys


@pytest.mark.parametrize("method,kind,inner", [("minres", "diag", "exact"), ("minres", "diag", "pcg"),
                                               ("fgmres", "diag", "exact"), ("fgmres", "tri", "exact"),
                                               ("fgmres", "tri", "pcg")])
def test_krylov_matches_direct(small_system, method, kind, inner):
    sys = small_system
    ud, pd = solvers.solve_direct(sys)
    u, p, res = solvers.solve_krylov(sys, method, kind, inner, rtol=1e-12, inner_rtol=1e-14)
    assert res.converged and res.relres <= 1e-12
    np.testing.assert_allclose(u, ud, atol=1e-9 * np.abs(ud).max())
    np.testing.assert_allclose(p, pd, atol=1e-9 * np.abs(pd).max())


def test_krylov_random_rhs_and_scipy(small_system):
    """Random RHS (no special structure): our MINRES and FGMRES reach 1e-10 and
    agree with SciPy's MINRES using the same preconditioner."""
    sys = small_system
    rng = np.random.default_rng(5)
    b = rng.standard_normal(sys.n)
    A = sys.saddle()
    P = solvers.BlockPreconditioner(sys, "diag", "exact")
    r1 = solvers.minres(A, b, P, rtol=1e-10)
    r2 = solvers.fgmres(A, b, solvers.BlockPreconditioner(sys, "tri", "exact"), 30, rtol=1e-10)
    Pop = spla.LinearOperator(A.shape, matvec=P)
    xs, info = spla.minres(A, b, M=Pop, rtol=1e-13, maxiter=5000)
    xd = spla.spsolve(A.tocsc(), b)
    assert r1.converged and r2.converged
    for x in (r1.x, r2.x, xs):
        assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    assert 10 < r1.iters < 1000


def test_pcg_matches_direct(small_system):
    S = solvers.schur(small_system)
    rng = np.random.default_rng(2)
    b = rng.standard_normal(S.shape[0])
    res = solvers.pcg(S, b, rtol=1e-13)
    assert res.converged
    np.testing.assert_allclose(res.x, spla.spsolve(S.tocsc(), b), rtol=1e-10, atol=1e-12)


def _unit_cube_l2_sq(a0, a):
    """int over [0,1]^3 of (a0 + a.x)^2, expanded by hand."""
    a = np.asarray(a, float)
    cross = sum(a[i] * a[j] for i in range(3) for j in range(i + 1, 3))
    return a0 * a0 + a0 * a.sum() + (a * a).sum() / 3.0 + cross / 2.0


def test_indicators_on_the_linear_patch():
    """Linear p = a0 + a.x, K = 1, on 3^3 cubes.  The paper's k = 1 element
    reproduces the constant flux, so e_v vanishes; its P0 pressure is the
    cell mean p(x_P), so e_q^2 ||p||^2 = sum_P int_P (a.(x - x_P))^2 =
    n^3 h^5 |a|^2 / 12 with h = 1/n.  The k = 2 element has P1 pressure and
    reproduces p, so both indicators vanish.  A mis-scaled or mis-signed term
    in either indicator fails one of these."""
    a0, a = 0.3, (1.0, -2.0, 0.5)
    prob = fields.linear_problem(a0, a)
    n = 3
    m = hex_mesh(n)
    nu = np.ones(m.n_cells)
    sys = assemble(m, paper_element(1), nu, f=prob.f, gD=prob.gD, keep_local=True)
    u, p = solvers.solve_direct(sys)
    ev, eq = errors.indicators(sys, sys.cells, sys.dofmap, u, p, prob.u, prob.p, nu)
    h = 1.0 / n
    eq_exact = np.sqrt(n ** 3 * h ** 5 * np.dot(a, a) / 12.0 / _unit_cube_l2_sq(a0, a))
    assert ev <= 1e-12
    assert eq == pytest.approx(eq_exact, rel=1e-10)
    sys2 = assemble(m, paper_element(2), nu, f=prob.f, gD=prob.gD, keep_local=True)
    u2, p2 = solvers.solve_direct(sys2)
    ev2, eq2 = errors.indicators(sys2, sys2.cells, sys2.dofmap, u2, p2, prob.u, prob.p, nu)
    assert ev2 <= 1e-11 and eq2 <= 1e-11
