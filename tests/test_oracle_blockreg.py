"""Pins for the oracle's Block-Reg preconditioner (paper Sec. 5: block-diagonal
with an AMG of A + B^T W^-1 B for the flux block and W^-1 for the pressure
block, W = gamma I, gamma = h^2 with h the mean cell diameter of eq. meshSize)
and for the Chebyshev smoother of its AMG cycle."""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import E0, amg, assemble, paper_element, solvers
from synth import fields, hex_mesh, prism_mesh, tet_mesh
from synth.voronoi import voronoi_mesh


@pytest.mark.parametrize("make", [hex_mesh, tet_mesh, prism_mesh], ids=["hex", "tet", "prism"])
@pytest.mark.parametrize("n", [2, 3])
def test_mesh_size_structured(make, n):
    """Every cell of these grids contains a main diagonal of its cube and no
    longer segment: h_P = sqrt(3)/n for all cells, so h = sqrt(3)/n."""
    m = make(n)
    sys_ = assemble(m, E0, np.ones(m.n_cells))
    assert solvers.mesh_size(sys_) == pytest.approx(np.sqrt(3.0) / n, rel=1e-14)


def test_mesh_size_voronoi_brute_force():
    """h = mean over cells of the largest distance between two vertices of
    the cell, computed here directly from the vertex coordinates."""
    m = voronoi_mesh(25, seed=4, lloyd=2)
    sys_ = assemble(m, E0, np.ones(m.n_cells))
    hs = []
    for c in range(m.n_cells):
        vs = np.unique(np.concatenate([m.face_vertices(f) for f in m.cell_faces(c)]))
        X = m.xyz[vs]
        hs.append(np.sqrt(((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)).max())
    assert solvers.mesh_size(sys_) == pytest.approx(np.mean(hs), rel=1e-13)


def _bc_neumann(m):
    m.face_bc = np.where(m.face_bc != 0, 2, 0).astype(np.int8)
    return m


@pytest.mark.parametrize("spec", [E0, paper_element(1)], ids=["E0", "K1"])
@pytest.mark.parametrize("neumann", [False, True], ids=["dirichlet", "flux"])
def test_regularized_is_cellwise_sum(spec, neumann):
    """A + B^T W^-1 B = sum_P (nu_P M_P + B_P^T B_P / gamma) assembled from
    the local matrices (B^T B couples only DOFs of one cell, as the pressure
    DOFs of P belong to P alone); prescribed-flux DOFs keep a unit row."""
    m = voronoi_mesh(20, seed=2, lloyd=2)
    if neumann:
        m = _bc_neumann(m)
    prob = fields.paper_polynomial_problem()
    K = fields.K_lognormal(m.n_cells, seed=1)
    sys_ = assemble(m, spec, 1.0 / K, f=prob.f, flux=prob.u if neumann else None, keep_local=True)
    gamma = 0.37
    A = solvers.regularized(sys_, gamma).toarray()
    R = np.zeros((sys_.n_u, sys_.n_u))
    for loc, dm in zip(sys_.local, sys_.dofmap):
        R[np.ix_(dm, dm)] += loc["M"] + loc["B"].T @ loc["B"] / gamma
    if neumann:
        fx = sys_.fixed
        assert fx.size > 0
        R[fx, :] = 0.0
        R[:, fx] = 0.0
        R[fx, fx] = 1.0
    np.testing.assert_allclose(A, R, rtol=0, atol=1e-13 * np.abs(R).max())


@pytest.mark.parametrize("spec", [E0, paper_element(1)], ids=["E0", "K1"])
def test_exact_block_reg_spectrum(spec):
    """With the flux block inverted exactly, P = diag(A + B^T B / gamma,
    gamma I) and K = [A B^T; B 0] give K x = mu P x with mu = 1 (n_u times:
    x = (u, B u / gamma)) and mu = -kappa / (kappa + gamma) for every
    eigenvalue kappa of the exact Schur complement B A^-1 B^T (from
    (1 - mu)(A + (1 + mu) B^T B / (mu gamma)) u = 0)."""
    m = hex_mesh(2) if spec is E0 else prism_mesh(1)
    prob = fields.sine_problem()
    sys_ = assemble(m, spec, 1.0 / fields.K_lognormal(m.n_cells, seed=3), f=prob.f, gD=prob.gD)
    gamma = 0.05
    Kd = sys_.saddle().toarray()
    Ar = solvers.regularized(sys_, gamma).toarray()
    P = sla.block_diag(Ar, gamma * np.eye(sys_.n_p))
    mu = np.sort(sla.eigvals(Kd, P).real)
    Ad, Bd = sys_.M.toarray(), sys_.B.toarray()
    kappa = sla.eigvalsh(Bd @ np.linalg.solve(Ad, Bd.T))
    ref = np.sort(np.concatenate([np.ones(sys_.n_u), -kappa / (kappa + gamma)]))
    np.testing.assert_allclose(mu, ref, atol=1e-9)


def _small_spd(n, seed):
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.diag(rng.uniform(0.5, 2.0, n))
    return sp.csr_matrix(A)


@pytest.mark.parametrize("degree", [1, 2, 3])
def test_chebyshev_error_factors(degree):
    """Chebyshev smoothing from zero leaves the error p(lambda) v on every
    generalised eigenvector A v = lambda D v, p(l) = T_k((theta - l)/delta) /
    T_k(theta/delta) on [lo, hi] = [rho/10, rho] (T_k the Chebyshev
    polynomial of the first kind)."""
    A = _small_spd(24, 5)
    H = amg.setup(A, coarse_max=100, smoother="chebyshev", degree=degree)
    lv = H.levels[0]
    D = A.diagonal()
    lam, V = sla.eigh(A.toarray(), np.diag(D))
    hi = amg.gershgorin_rho(A)
    lo = hi / 10.0
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    T = {1: lambda t: t, 2: lambda t: 2 * t * t - 1, 3: lambda t: 4 * t ** 3 - 3 * t}[degree]
    assert lam.max() <= hi * (1 + 1e-12)
    for i in range(0, 24, 5):
        v = V[:, i]
        x = amg.chebyshev(lv, A @ v, np.zeros(24), degree)
        p = T((th - lam[i]) / de) / T(th / de)
        np.testing.assert_allclose(v - x, p * v, atol=1e-12 * np.abs(v).max())
        assert abs(p) < 1.0


@pytest.mark.parametrize("smoother", ["jacobi", "chebyshev"])
def test_cycle_symmetric_positive_definite(smoother):
    """The V-cycle matrix (the cycle applied to the unit vectors) of the
    regularised flux operator is symmetric and positive definite, so it can
    precondition MINRES."""
    m = hex_mesh(4)
    sys_ = assemble(m, E0, np.ones(m.n_cells))
    Ar = solvers.regularized(sys_, solvers.mesh_size(sys_) ** 2)
    H = amg.setup(Ar, coarse_max=16, smoother=smoother)
    assert len(H.levels) >= 2
    n = Ar.shape[0]
    C = np.column_stack([amg.vcycle(H, e) for e in np.eye(n)])
    np.testing.assert_allclose(C, C.T, atol=1e-12 * np.abs(C).max())
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0.0


def test_chebyshev_cycle_beats_jacobi_cycle():
    """Two Chebyshev steps per smoothing contract the regularised flux
    operator's error faster than one damped-Jacobi step (the paper's GAMG
    default against the plain V(1,1) cycle)."""
    m = hex_mesh(6)
    sys_ = assemble(m, paper_element(1), np.ones(m.n_cells))
    Ar = solvers.regularized(sys_, solvers.mesh_size(sys_) ** 2)
    rng = np.random.default_rng(0)
    e0 = rng.standard_normal(Ar.shape[0])
    rates = {}
    for sm in ("jacobi", "chebyshev"):
        H = amg.setup(Ar, smoother=sm)
        e = e0.copy()
        for _ in range(5):
            e = e - amg.vcycle(H, Ar @ e)
        rates[sm] = np.sqrt(e @ (Ar @ e)) / np.sqrt(e0 @ (Ar @ e0))
    assert rates["chebyshev"] < 0.5 * rates["jacobi"], rates


@pytest.mark.parametrize("spec", [E0, paper_element(1)], ids=["E0", "K1"])
@pytest.mark.parametrize("method", ["minres", "fgmres"])
@pytest.mark.parametrize("neumann", [False, True], ids=["dirichlet", "flux"])
def test_block_reg_reaches_direct_solution(spec, method, neumann):
    m = hex_mesh(4)
    if neumann:
        m = _bc_neumann(m)
    prob = fields.paper_polynomial_problem()
    sys_ = assemble(m, spec, np.ones(m.n_cells), f=prob.f, gD=prob.gD, flux=prob.u if neumann else None)
    u, p, res = solvers.solve_krylov(sys_, method, "reg", rtol=1e-11, restart=30, maxit=3000)
    ud, pd = solvers.solve_direct(sys_)
    assert res.converged
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-8 * np.linalg.norm(pd)
