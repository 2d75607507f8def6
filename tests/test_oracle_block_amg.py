"""Pins for oracle/block_amg.py: smoothed aggregation on point blocks --
the cell blocks of the k = 2 Schur block (four P1 pressure moments per
cell, eq. presMom, near-null space the moments of 1, x, y, z), and the face
and cell blocks of Block-Reg's regularised flux block A_reg (near-null
space the DOFs of the constant fields), directly at k = 1 and behind the
cell-wise condensation of the interior DOFs at k = 1 and 2."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import E0, amg, assemble, block_amg, paper_element, solvers
from synth import fields, hex_mesh
from synth.voronoi import voronoi_mesh

K2 = paper_element(2)


def _k2_schur(m, seed=None, **kw):
    nu = np.ones(m.n_cells) if seed is None else 1.0 / fields.K_lognormal(m.n_cells, seed=seed, sigma=0.5)
    sys_ = assemble(m, K2, nu, keep_local=True, **kw)
    return sys_, solvers.schur(sys_).tocsr()


def test_unit_blocks_give_the_scalar_strength_and_aggregates():
    """With 1 x 1 blocks the block norm is |a_ij| and the rule reduces to the
    scalar strength of oracle/amg.py (the same neighbour set per row, listed
    in column order), hence the same aggregates."""
    m = voronoi_mesh(60, seed=2, lloyd=2)
    sys_ = assemble(m, E0, 1.0 / fields.K_lognormal(m.n_cells, seed=1))
    S = solvers.schur(sys_)
    for theta in (0.08, 0.25):
        p1, i1 = block_amg.block_strength(S, 1, theta)
        p0, i0 = amg.strength(S, theta)
        np.testing.assert_array_equal(p1, p0)
        for r in range(S.shape[0]):
            np.testing.assert_array_equal(i1[p1[r]:p1[r + 1]], np.sort(i0[p0[r]:p0[r + 1]]))
    a1 = amg.aggregate(S.shape[0], p1, i1)
    a0 = amg.aggregate(S.shape[0], p0, i0)
    np.testing.assert_array_equal(a1[0], a0[0])


def test_block_norms_brute_force():
    _, S = _k2_schur(hex_mesh(2), seed=3)
    N = block_amg.block_norms(S, 4).toarray()
    D = S.toarray()
    for I in range(8):
        for J in range(8):
            assert N[I, J] == pytest.approx(np.linalg.norm(D[4 * I:4 * I + 4, 4 * J:4 * J + 4]), rel=1e-14, abs=0)


def test_pressure_modes_on_cubes():
    """Cube cells of side a (h_P = sqrt(3) a, m_x = (x - x_P)/h_P): the
    moments of 1 are (1, 0, 0, 0); those of x are (x_P, a / (12 sqrt 3), 0,
    0) since (1/|P|) int (x - x_P)^2 = a^2 / 12 and the mixed central
    moments vanish; likewise for y and z."""
    n = 3
    a = 1.0 / n
    m = hex_mesh(n)
    sys_ = assemble(m, K2, np.ones(m.n_cells), keep_local=True)
    B = block_amg.pressure_modes(sys_)
    c = a / (12.0 * np.sqrt(3.0))
    for P, cell in enumerate(sys_.cells):
        blk = B[4 * P:4 * P + 4]
        np.testing.assert_allclose(blk[:, 0], [1, 0, 0, 0], atol=1e-14)
        for d in range(3):
            ref = np.zeros(4)
            ref[0] = cell.centroid[d]
            ref[1 + d] = c
            np.testing.assert_allclose(blk[:, 1 + d], ref, atol=1e-14)


def test_constant_mode_is_the_kernel_with_flux_data():
    """With flux data on the whole boundary S has the constant pressure as
    its kernel (B^T applied to it vanishes on the free flux DOFs), and the
    first mode is that vector."""
    m = hex_mesh(3, bc=2)
    prob = fields.paper_polynomial_problem()
    sys_, S = _k2_schur(m, seed=2, f=prob.f, flux=prob.u)
    B = block_amg.pressure_modes(sys_)
    np.testing.assert_allclose(B[:, 0], sys_.null_vec, atol=1e-13)
    assert np.abs(S @ B[:, 0]).max() <= 1e-12 * abs(S).max()


def test_start_vector_from_splitmix64():
    """v_i = 2 (splitmix64(i) >> 11) / 2^53 - 1: v_0 from SplitMix64's
    published first output (counter 0), the rest in [-1, 1) with mean near
    zero."""
    v = block_amg.start_vector(1000)
    assert v[0] == 2.0 * (0xE220A8397B1DCDAF >> 11) / 2.0 ** 53 - 1.0
    assert v[7] == 2.0 * (amg.splitmix64(7) >> 11) / 2.0 ** 53 - 1.0
    assert np.all((v >= -1.0) & (v < 1.0)) and abs(v.mean()) < 0.1


@pytest.mark.parametrize("mesh", ["hex", "cvt"])
def test_spectral_estimate(mesh):
    """C = L^-1 S L^-T has the spectrum of D^-1 S; its Gershgorin bound lies
    above lambda_max, the Lanczos Ritz value below it and within 10% after
    10 steps, and the estimate rho gives a convergent smoother
    (2/3 lambda_max < rho <= Gershgorin)."""
    m = hex_mesh(5) if mesh == "hex" else voronoi_mesh(150, seed=5, lloyd=5)
    _, S = _k2_schur(m, seed=4)
    C = block_amg.symmetric_form(S, 4)
    lam = np.linalg.eigvalsh(C.toarray())
    D = (block_amg.block_diag_inv(S, 4) @ S).toarray()
    np.testing.assert_allclose(np.sort(np.linalg.eigvals(D).real), lam, rtol=1e-9, atol=1e-12)
    gersh = float(np.asarray(abs(C).sum(axis=1)).max())
    theta = block_amg.lanczos_max(C, 10)
    rho = block_amg.rho_estimate(S, 4)
    assert theta <= lam.max() * (1 + 1e-12)
    assert theta >= 0.9 * lam.max()
    assert gersh >= lam.max()
    assert 2.0 / 3.0 * lam.max() < rho <= gersh
    assert gersh > 1.4 * lam.max()          # why the plain bound is not used


def test_tentative_prolongator():
    """T has orthonormal columns, reproduces the near-null space exactly
    (T B_c = B), couples each aggregate's DOFs only to its own columns, and
    B_c is upper triangular per aggregate with a positive diagonal."""
    m = voronoi_mesh(80, seed=3, lloyd=3)
    sys_, S = _k2_schur(m, seed=1)
    B = block_amg.pressure_modes(sys_)
    ptr, idx = block_amg.block_strength(S, 4, 0.08)
    agg, nc = amg.aggregate(m.n_cells, ptr, idx)
    assert 0 < nc < m.n_cells
    T, Bc = block_amg.tentative(agg, nc, B, 4)
    np.testing.assert_allclose((T.T @ T).toarray(), np.eye(4 * nc), atol=1e-13)
    keep = np.repeat(agg >= 0, 4)
    np.testing.assert_allclose(T @ Bc, B * keep[:, None], atol=1e-13 * np.abs(B).max())
    Tc = T.tocoo()
    assert np.all(agg[Tc.row // 4] == Tc.col // 4)
    for a in range(nc):
        R = Bc[4 * a:4 * a + 4]
        np.testing.assert_array_equal(np.tril(R, -1), 0.0)
        assert np.all(np.diag(R) > 0.0)


def test_rank_deficient_aggregates_dissolved():
    """Aggregates on which the near-null space loses rank (two blocks
    spanning only two of three modes, a zero mode) leave the coarse space,
    the others keep their order; the decision agrees with the SVD rank on
    random full-rank and exactly rank-deficient blocks, including badly
    scaled full-rank ones (singular value ratio 1e-3)."""
    rng = np.random.default_rng(4)
    bs, m = 3, 3
    full = rng.standard_normal((2 * bs, m))
    two = rng.standard_normal((2 * bs, 2)) @ np.array([[1.0, 0.0, 1.0], [0.0, 1.0, 1.0]])
    zero = rng.standard_normal((2 * bs, m))
    zero[:, 1] = 0.0
    U, _, Vt = np.linalg.svd(rng.standard_normal((2 * bs, m)), full_matrices=False)
    scaled = U @ np.diag([1.0, 1e-2, 1e-3]) @ Vt
    B = np.vstack([full, two, zero, scaled, rng.standard_normal((bs, m))])
    agg = np.array([0, 0, 1, 1, 2, 2, 3, 3, -1])
    new, nc = block_amg.dissolve_rank_deficient(agg, 4, B, bs)
    np.testing.assert_array_equal(new, [0, 0, -1, -1, -1, -1, 1, 1, -1])
    assert nc == 2
    for a, blk in enumerate((full, two, zero, scaled)):
        assert (np.linalg.matrix_rank(blk) == m) == (a in (0, 3))
    T, Bc = block_amg.tentative(new, nc, B, bs)
    keep = np.repeat(new >= 0, bs)
    np.testing.assert_allclose(T @ Bc, B * keep[:, None], atol=1e-13)
    # nothing changes where every aggregate has full rank
    same, nc2 = block_amg.dissolve_rank_deficient(np.array([0, 0, 1, 1, -1]), 2,
                                                  np.vstack([full, scaled, B[-bs:]]), bs)
    np.testing.assert_array_equal(same, [0, 0, 1, 1, -1])
    assert nc2 == 2


def test_cycle_symmetric_positive_definite():
    _, S = _k2_schur(hex_mesh(4), seed=6)
    H = block_amg.setup(S, 4, block_amg.pressure_modes(_k2_schur(hex_mesh(4), seed=6)[0]), coarse_max=4)
    assert len(H.levels) >= 2 and H.levels[1].bs == 4
    n = S.shape[0]
    C = np.column_stack([block_amg.vcycle(H, e) for e in np.eye(n)])
    np.testing.assert_allclose(C, C.T, atol=1e-12 * np.abs(C).max())
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0.0


def test_coarse_correction_is_an_S_orthogonal_projector():
    sys_, S = _k2_schur(hex_mesh(4), seed=7)
    H = block_amg.setup(S, 4, block_amg.pressure_modes(sys_), coarse_max=4)
    P = H.levels[0].P.toarray()
    Sd = S.toarray()
    E = np.eye(S.shape[0]) - P @ np.linalg.solve(P.T @ Sd @ P, P.T @ Sd)
    np.testing.assert_allclose(E @ E, E, atol=1e-10)
    np.testing.assert_allclose(Sd @ E, (Sd @ E).T, atol=1e-10 * np.abs(Sd).max())


@pytest.mark.slow
@pytest.mark.parametrize("mesh", ["hex6", "hex8", "cvt400"])
def test_block_amg_iterations_bounded(mesh):
    """Block-AMG-PCG on the k = 2 Schur block: at most 22 iterations to 1e-8
    for a random right-hand side on these meshes, under half of Jacobi-PCG's
    and of the scalar AMG's (which keeps neither the cell blocks nor the
    linear modes together)."""
    m = {"hex6": lambda: hex_mesh(6), "hex8": lambda: hex_mesh(8),
         "cvt400": lambda: voronoi_mesh(400, seed=7, lloyd=10)}[mesh]()
    sys_, S = _k2_schur(m)
    b = np.random.default_rng(0).standard_normal(S.shape[0])
    H = block_amg.setup(S, 4, block_amg.pressure_modes(sys_))
    rb = block_amg.pcg(S, b, H, rtol=1e-8)
    rj = solvers.pcg(S, b, rtol=1e-8)
    rs = amg.amg_pcg(S, b, amg.setup(S), rtol=1e-8)
    assert rb.converged and rb.relres <= 1e-7
    assert rb.iters <= 22, rb.iters
    assert 2 * rb.iters < rj.iters and 2 * rb.iters < rs.iters, (rb.iters, rj.iters, rs.iters)


@pytest.mark.parametrize("flux", [False, True], ids=["dirichlet", "flux"])
def test_krylov_with_block_amg_reaches_direct_solution(flux):
    """k = 2 Block-Schur FGMRES with the Schur block solved by block-AMG-PCG
    reaches the direct solution, also with the mean-zero multiplier."""
    prob = fields.paper_polynomial_problem()
    m = hex_mesh(3, bc=2 if flux else 1)
    nu = 1.0 / fields.K_lognormal(m.n_cells, seed=5, sigma=0.5)
    if flux:
        sys_ = assemble(m, K2, nu, f=prob.f, flux=prob.u, keep_local=True)
    else:
        sys_ = assemble(m, K2, nu, f=prob.f, gD=prob.gD, keep_local=True)
    ud, pd = solvers.solve_direct(sys_)
    for kind in ("diag", "tri"):
        u, p, res = solvers.solve_krylov(sys_, "fgmres", kind, "block-amg", rtol=1e-11, inner_rtol=1e-13)
        assert res.converged
        np.testing.assert_allclose(u, ud, atol=1e-8 * np.abs(ud).max())
        np.testing.assert_allclose(p, pd, atol=1e-8 * np.abs(pd).max())


def test_block_amg_with_p0_pressure():
    """With one pressure DOF per cell (K1) the same code runs on 1 x 1 blocks
    with the constant as the only near-null vector."""
    m = hex_mesh(4)
    prob = fields.sine_problem()
    sys_ = assemble(m, paper_element(1), np.ones(m.n_cells), f=prob.f, gD=prob.gD, keep_local=True)
    assert block_amg.pressure_modes(sys_).shape == (m.n_cells, 1)
    ud, pd = solvers.solve_direct(sys_)
    u, p, res = solvers.solve_krylov(sys_, "fgmres", "tri", "block-amg", rtol=1e-11, inner_rtol=1e-13)
    assert res.converged
    np.testing.assert_allclose(p, pd, atol=1e-8 * np.abs(pd).max())


# ---- the same construction on the regularised flux block of Block-Reg (k = 1)

def test_flux_modes_on_cubes():
    """The constant field e_x has face moments (1, 0, 0) on x-normal faces
    (global normal +x, centred face monomials) and 0 on the others, and zero
    cross moments (int_P (x - x_P) = 0); likewise for e_y, e_z."""
    n = 2
    m = hex_mesh(n)
    sys_ = assemble(m, paper_element(1), np.ones(m.n_cells), keep_local=True)
    B = block_amg.flux_modes(sys_)
    nfx = n * n * (n + 1)                     # faces per normal direction, x first
    ref = np.zeros_like(B)
    for d in range(3):
        for f in range(d * nfx, (d + 1) * nfx):
            ref[3 * f, d] = 1.0
    np.testing.assert_allclose(B, ref, atol=1e-13)


def test_block_chebyshev_error_factors():
    """Block-Chebyshev smoothing from zero leaves the error p(lambda) v on
    every generalised eigenvector A v = lambda D v of the block diagonal D,
    p(l) = T_2((theta - l)/delta) / T_2(theta/delta) on [rho/10, rho]."""
    m = hex_mesh(2)
    sys_ = assemble(m, paper_element(1), np.ones(m.n_cells), keep_local=True)
    A = solvers.regularized(sys_, 0.3)
    H = block_amg.setup(A, 3, block_amg.flux_modes(sys_), coarse_max=1000, smoother="chebyshev")
    lv = H.levels[0]
    D = np.linalg.inv(lv.Dinv.toarray())
    import scipy.linalg as sla
    lam, V = sla.eigh(A.toarray(), D)
    hi, lo = lv.rho, lv.rho / 10.0
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    assert lam.max() < 1.5 * hi
    for i in range(0, lam.size, 7):
        v = V[:, i]
        x = block_amg.chebyshev(lv, A @ v, np.zeros(v.size), 2)
        t = (th - lam[i]) / de
        p = (2 * t * t - 1) / (2 * (th / de) ** 2 - 1)
        np.testing.assert_allclose(v - x, p * v, atol=1e-11 * np.abs(v).max())


def test_block_chebyshev_cycle_spd_on_areg():
    m = voronoi_mesh(30, seed=4, lloyd=3)
    sys_ = assemble(m, paper_element(1), np.ones(m.n_cells), keep_local=True)
    A = solvers.regularized(sys_, solvers.mesh_size(sys_) ** 2)
    H = block_amg.setup(A, 3, block_amg.flux_modes(sys_), coarse_max=8, smoother="chebyshev")
    assert len(H.levels) >= 2 and H.levels[1].bs == 3
    n = A.shape[0]
    C = np.column_stack([block_amg.vcycle(H, e) for e in np.eye(n)])
    np.testing.assert_allclose(C, C.T, atol=1e-12 * np.abs(C).max())
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0.0


@pytest.mark.parametrize("case", ["hex-flux", "voronoi-dirichlet"])
def test_block_reg_with_block_amg_reaches_direct_solution(case):
    prob = fields.paper_polynomial_problem()
    if case == "hex-flux":
        m = hex_mesh(3, bc=2)
        kw = dict(f=prob.f, flux=prob.u)
    else:
        m = voronoi_mesh(40, seed=3, lloyd=3)
        kw = dict(f=prob.f, gD=prob.gD)
    sys_ = assemble(m, paper_element(1), np.ones(m.n_cells), keep_local=True, **kw)
    ud, pd = solvers.solve_direct(sys_)
    u, p, res = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-11, restart=30, maxit=3000,
                                     reg_smoother="block-chebyshev")
    assert res.converged
    np.testing.assert_allclose(u, ud, atol=1e-8 * np.abs(ud).max())
    np.testing.assert_allclose(p, pd, atol=1e-8 * np.abs(pd).max())


@pytest.mark.slow
def test_block_amg_on_areg_cuts_block_reg_counts_on_cvt():
    """k = 1 on 125 CVT cells: Block-Reg FGMRES(30) to 1e-6 with the point-
    block AMG of A_reg takes under half the iterations of the scalar
    Chebyshev cycle (41 against 162 when written)."""
    m = voronoi_mesh(125, seed=7, lloyd=10)
    prob = fields.paper_polynomial_problem()
    sys_ = assemble(m, paper_element(1), np.ones(m.n_cells), f=prob.f, gD=prob.gD, keep_local=True)
    _, _, rs = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-6, restart=30, maxit=2000)
    _, _, rb = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-6, restart=30, maxit=2000,
                                    reg_smoother="block-chebyshev")
    assert rb.converged and rb.iters <= 50
    assert 2 * rb.iters < rs.iters, (rb.iters, rs.iters)


# ---- Block-Reg's A_reg with the interior DOFs condensed (k = 1 and 2)

def test_condensed_cycle_is_exact_with_an_exact_face_solve(monkeypatch):
    """Eliminating the interior DOFs cell by cell is exact: with the face
    system solved exactly the cycle returns A_reg^-1 r."""
    import scipy.sparse.linalg as spla
    m = voronoi_mesh(20, seed=2, lloyd=2)
    sys_ = assemble(m, K2, 1.0 / fields.K_lognormal(m.n_cells, seed=2, sigma=0.5), keep_local=True)
    A = solvers.regularized(sys_, 0.2)
    cc = block_amg.CondensedCycle(sys_, A)
    assert cc.Sf.shape[0] == K2.nfd * m.n_faces
    monkeypatch.setattr(block_amg, "vcycle", lambda H, b: spla.spsolve(cc.Sf.tocsc(), b))
    r = np.random.default_rng(1).standard_normal(A.shape[0])
    ref = spla.spsolve(A.tocsc(), r)
    np.testing.assert_allclose(cc(r), ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_condensed_cycle_spd():
    m = hex_mesh(3)
    sys_ = assemble(m, K2, np.ones(m.n_cells), keep_local=True)
    A = solvers.regularized(sys_, solvers.mesh_size(sys_) ** 2)
    cc = block_amg.CondensedCycle(sys_, A)
    n = A.shape[0]
    C = np.column_stack([cc(e) for e in np.eye(n)])
    np.testing.assert_allclose(C, C.T, atol=1e-11 * np.abs(C).max())
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0.0


@pytest.mark.parametrize("case", ["k2-hex-flux", "k2-voronoi", "k1-voronoi-flux"])
def test_block_reg_condensed_reaches_direct_solution(case):
    prob = fields.paper_polynomial_problem()
    spec = K2 if case.startswith("k2") else paper_element(1)
    flux = case.endswith("flux")
    m = hex_mesh(3, bc=2) if "hex" in case else voronoi_mesh(40, seed=3, lloyd=3)
    if flux and "voronoi" in case:
        m.face_bc = np.where(m.face_bc != 0, 2, 0).astype(np.int8)
    kw = dict(f=prob.f, flux=prob.u) if flux else dict(f=prob.f, gD=prob.gD)
    sys_ = assemble(m, spec, np.ones(m.n_cells), keep_local=True, **kw)
    ud, pd = solvers.solve_direct(sys_)
    u, p, res = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-11, restart=30, maxit=3000,
                                     reg_smoother="condensed-block")
    assert res.converged
    np.testing.assert_allclose(u, ud, atol=1e-8 * np.abs(ud).max())
    np.testing.assert_allclose(p, pd, atol=1e-8 * np.abs(pd).max())


@pytest.mark.slow
def test_condensed_block_reg_on_cvt_k2():
    """k = 2, flux data, 27 CVT cells: Block-Reg to 1e-6 with the condensed
    point-block cycle takes under 100 iterations and under half the count
    of the edge-patch Schwarz variant (407 when written; the paper's GAMG
    count on its 27-cell CVT mesh is 151)."""
    prob = fields.paper_polynomial_problem()
    m = voronoi_mesh(27, seed=7, lloyd=10)
    m.face_bc = np.where(m.face_bc != 0, 2, 0).astype(np.int8)
    sys_ = assemble(m, K2, np.ones(m.n_cells), f=prob.f, flux=prob.u, keep_local=True)
    _, _, rc = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-6, restart=30, maxit=2000,
                                    reg_smoother="condensed-block")
    _, _, re = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-6, restart=30, maxit=2000,
                                    reg_smoother="edge-schwarz", mesh=m)
    assert rc.converged and rc.iters < 100, rc.iters
    assert 2 * rc.iters < re.iters, (rc.iters, re.iters)


def test_cholesky_qr_gives_the_same_factor():
    """The thin QR with R_jj > 0 is unique, so R = chol(B^T B)^T and
    Q = B R^-1 (Cholesky-QR, the form a thread per aggregate computes)
    agree with the Householder factors on every aggregate of a k = 2
    Schur block."""
    m = voronoi_mesh(60, seed=4, lloyd=3)
    sys_, S = _k2_schur(m, seed=2)
    B = block_amg.pressure_modes(sys_)
    ptr, idx = block_amg.block_strength(S, 4, 0.08)
    agg, nc = amg.aggregate(m.n_cells, ptr, idx)
    for a in range(nc):
        members = np.nonzero(agg == a)[0]
        X = B[(members[:, None] * 4 + np.arange(4)[None, :]).ravel()]
        Q, R = block_amg.qr_positive(X)
        Rc = np.linalg.cholesky(X.T @ X).T
        np.testing.assert_allclose(Rc, R, rtol=0, atol=1e-9 * np.abs(R).max())
        np.testing.assert_allclose(X @ np.linalg.inv(Rc), Q, rtol=0, atol=1e-8)


def test_block_reg_condensed_with_minres():
    """The condensed cycle is symmetric positive definite, so Block-Reg with
    it also preconditions MINRES (k = 2, pressure data)."""
    prob = fields.paper_polynomial_problem()
    m = hex_mesh(3)
    sys_ = assemble(m, K2, np.ones(m.n_cells), f=prob.f, gD=prob.gD, keep_local=True)
    ud, pd = solvers.solve_direct(sys_)
    u, p, res = solvers.solve_krylov(sys_, "minres", "reg", rtol=1e-11, maxit=3000, reg_smoother="condensed-block")
    assert res.converged
    np.testing.assert_allclose(u, ud, atol=1e-8 * np.abs(ud).max())
    np.testing.assert_allclose(p, pd, atol=1e-8 * np.abs(pd).max())
