"""Parity of the paper's k = 2 element matrices (Sec. 4.1-4.3 at k = 2: six
face moments, three gradient and eleven cross moments, P1 pressure) between
the CUDA element kernel and the oracle's local system, cell by cell, on hex,
sheared hex, tet, prism, Octa and Voronoi meshes; the assembled saddle-point
matrix, right-hand side and Schur approximation; solves against the
oracle's direct solve; and the combinations that are not built for k = 2."""

import numpy as np
import pytest

from oracle import paper_element
from oracle.element import local_system
from oracle.assemble import mesh_cells
from synth import affine, fields, hex_mesh, octa_mesh, prism_mesh, tet_mesh
from synth.voronoi import voronoi_mesh

pytestmark = pytest.mark.gpu

A_SHEAR = np.array([[1.0, 0.3, 0.1], [0.0, 0.8, -0.2], [0.1, 0.0, 1.2]])
MESHES = {
    "hex3": lambda: hex_mesh(3),
    "sheared": lambda: affine(hex_mesh(2), A_SHEAR, (0.1, 0.0, -0.3)),
    "tet2": lambda: tet_mesh(2),
    "prism2": lambda: prism_mesh(2),
    "octa2": lambda: octa_mesh(2),
    "cvt40": lambda: voronoi_mesh(40, seed=3, lloyd=5),
}
# Relative tolerance per cell (to the largest entry): the k = 2 projections
# solve the 10 x 10 Gram matrix of P_2 and the 6 x 6 face Gram matrices of
# M_2(f), whose conditioning on the Voronoi cells (small faces) costs a few
# more digits than at k = 1.
TOL = {"hex3": 1e-12, "sheared": 1e-11, "tet2": 1e-11, "prism2": 1e-11, "octa2": 1e-11, "cvt40": 1e-9}


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    import torch
    assert torch.cuda.is_available()
    return vemsolve


@pytest.mark.parametrize("mname", list(MESHES))
@pytest.mark.parametrize("reuse", [1, 0])
def test_k2_local_matrices(vs, mname, reuse):
    spec = paper_element(2)
    mesh = MESHES[mname]()
    K = fields.K_lognormal(mesh.n_cells, seed=3, sigma=1.0)
    s = vs.Solver(mesh, element=vs.VEM_ELEMENT_K2, reuse=reuse)
    try:
        s.set_coefficient(K)
        ms, ncls = s.assemble_local()
        loc = s.local_matrices()
        n_u, n_p = s.sizes()
    finally:
        s.close()
    assert n_u == spec.nfd * mesh.n_faces + spec.nid * mesh.n_cells
    assert n_p == spec.nq * mesh.n_cells
    assert ncls >= 1 and ms > 0.0
    cells = mesh_cells(mesh)
    for c, cell in enumerate(cells):
        ref = local_system(cell, spec, 1.0 / K[c])
        M, B = loc[c]
        assert M.shape == ref["M"].shape and B.shape == ref["B"].shape, c
        np.testing.assert_allclose(M, ref["M"], rtol=0, atol=TOL[mname] * np.abs(ref["M"]).max(),
                                   err_msg=f"cell {c}")
        np.testing.assert_allclose(B, ref["B"], rtol=0, atol=TOL[mname] * np.abs(ref["B"]).max(),
                                   err_msg=f"cell {c}")


def test_k2_switch_element(vs):
    """A handle switched between k = 2 and k = 1 solves both ways."""
    mesh = hex_mesh(2)
    prob = fields.quadratic_problem()
    s = vs.Solver(mesh, element=vs.VEM_ELEMENT_K2, krylov=1, precond=1, rtol=1e-11, inner_rtol=1e-13)
    try:
        s.set_data(prob.f, prob.gD)
        _, _, st2 = s.solve()
        s.set_options(element=vs.VEM_ELEMENT_K1)
        s.set_data(prob.f, prob.gD)
        _, _, st1 = s.solve()
        s.set_options(element=vs.VEM_ELEMENT_K2)
        s.set_data(prob.f, prob.gD)
        _, _, st3 = s.solve()
    finally:
        s.close()
    assert st1["relres"] <= 1e-11 and st2["relres"] <= 1e-11 and st3["relres"] <= 1e-11
    assert st2["n_p"] == 4 * mesh.n_cells and st1["n_p"] == mesh.n_cells


def _f2(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return 1.0 + X - 2.0 * Y * Y + X * Z


def _g2(x):
    X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
    return X * X - Y * Z + 0.5


# data of degree <= 2: the library's and the oracle's load rules are both
# exact for them, so the right-hand sides agree to rounding
SYS_MESHES = {"hex3": lambda: hex_mesh(3), "prism2": lambda: prism_mesh(2), "octa2": lambda: octa_mesh(2),
              "cvt30": lambda: voronoi_mesh(30, seed=4, lloyd=5)}
SYS_TOL = {"hex3": 1e-12, "prism2": 1e-11, "octa2": 1e-11, "cvt30": 1e-9}


def _k2_pair(vs, mname, **kw):
    from oracle import assemble
    mesh = SYS_MESHES[mname]()
    K = fields.K_lognormal(mesh.n_cells, seed=5, sigma=0.7)
    s = vs.Solver(mesh, element=vs.VEM_ELEMENT_K2, **kw)
    s.set_coefficient(K)
    s.set_data(_f2, _g2)
    sys_ = assemble(mesh, paper_element(2), 1.0 / K, f=_f2, gD=_g2)
    return s, sys_


@pytest.mark.parametrize("mname", list(SYS_MESHES))
def test_k2_saddle_rhs_and_schur(vs, mname):
    from oracle import solvers
    s, sys_ = _k2_pair(vs, mname)
    try:
        A, rhs = s.system()
        S, dM = s.schur()
    finally:
        s.close()
    Ar = sys_.saddle()
    assert A.shape == Ar.shape
    assert abs(A - Ar).max() <= SYS_TOL[mname] * abs(Ar).max()
    ref = sys_.rhs()
    np.testing.assert_allclose(rhs, ref, rtol=0, atol=SYS_TOL[mname] * np.abs(ref).max())
    Sr = solvers.schur(sys_)
    assert abs(S - Sr).max() <= SYS_TOL[mname] * abs(Sr).max()
    np.testing.assert_allclose(dM, sys_.M.diagonal(), rtol=SYS_TOL[mname] * 10)


@pytest.mark.parametrize("mname", ["hex3", "octa2", "cvt30"])
@pytest.mark.parametrize("krylov,prec,inner", [(0, 0, 0), (1, 1, 0), (1, 1, 1), (0, 0, 1)],
                         ids=["minres-diag-pcg", "fgmres-tri-pcg", "fgmres-tri-amg", "minres-diag-amg"])
def test_k2_solve_matches_direct(vs, mname, krylov, prec, inner):
    """(FGMRES(30) with the block-diagonal preconditioner stalls near 1e-8 on
    the Voronoi mesh at k = 2 -- the paper reports 600-700 GMRES iterations
    for Block-Schur on CVT meshes at k = 2 -- so the block-diagonal cases run
    MINRES, which is not restarted.  The block-triangular FGMRES(30) needs
    about 3,100 iterations there to 1e-12, a count that moves by a restart
    cycle with the rounding of the inner solves, so the cap is 6,000.)"""
    from oracle import solvers
    s, sys_ = _k2_pair(vs, mname, krylov=krylov, precond=prec, inner=inner, rtol=1e-12, inner_rtol=1e-13,
                       maxit=6000)
    try:
        u, p, st = s.solve()
    finally:
        s.close()
    ud, pd = solvers.solve_direct(sys_)
    assert st["relres"] <= 1e-12
    assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-9 * np.linalg.norm(pd)


def _cubic(K=1.0):
    """p in P_3, u = -K grad p in [P_2]^3, f = div u in P_1: every load and
    flux datum is integrated exactly by both sides' rules."""
    def p(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return X ** 3 - 2 * X * Y * Y + 0.5 * Z ** 3 + X * Y * Z + Y * Y - 0.4 * Z

    def u(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return -K * np.stack([3 * X * X - 2 * Y * Y + Y * Z, -4 * X * Y + X * Z + 2 * Y,
                              1.5 * Z * Z + X * Y - 0.4], 1)

    def f(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return -K * (2 * X + 2 + 3 * Z)

    return p, u, f


@pytest.mark.parametrize("mname", ["tet2", "prism2", "cvt30"])
def test_k2_cubic_dirichlet_patch(vs, mname):
    """Pressure data of a cubic p on the whole boundary, constant K: the
    library's solution is the interpolant of the exact flux and the P_1
    moments of p on triangular and Voronoi faces too -- the boundary term
    int_f g_D m^f has degree 5, which the k = 2 boundary rule (Radon's 7
    points per fan triangle) integrates exactly."""
    from oracle import assemble
    from oracle.element import interpolate
    from oracle.monomials import eval_mono3, mono3
    m = {"tet2": lambda: tet_mesh(2), "prism2": lambda: prism_mesh(2),
         "cvt30": lambda: voronoi_mesh(30, seed=4, lloyd=5)}[mname]()
    K = 1.7
    p_ex, u_ex, f_ex = _cubic(K)
    spec = paper_element(2)
    s = vs.Solver(m, element=vs.VEM_ELEMENT_K2, krylov=0, precond=0, rtol=1e-12, inner_rtol=1e-13, maxit=6000)
    try:
        assert s.quadrature_count(vs.VEM_QP_BFACE) == 7 * sum(
            int(m.face_vtx_ptr[f + 1] - m.face_vtx_ptr[f]) for f in np.nonzero(m.face_bc)[0])
        s.set_coefficient(np.full(m.n_cells, K))
        s.set_data(f_ex, p_ex)
        u, p, st = s.solve()
    finally:
        s.close()
    sys_ = assemble(m, spec, np.full(m.n_cells, 1.0 / K), keep_local=True)
    uI = np.zeros(sys_.n_u)
    for c, cell in enumerate(sys_.cells):
        uI[sys_.dofmap[c]] = interpolate(cell, spec, u_ex)
    pI = np.concatenate([(cell.qw * p_ex(cell.qp)) @ eval_mono3(mono3(1), cell.qp, cell.centroid, cell.diameter)
                         / cell.volume for cell in sys_.cells])
    assert st["relres"] <= 1e-12
    np.testing.assert_allclose(u, uI, atol=1e-9 * np.abs(uI).max())
    np.testing.assert_allclose(p, pI, atol=1e-9 * np.abs(pI).max())


def _flux_mesh(name):
    if name == "cvt30":
        m = voronoi_mesh(30, seed=4, lloyd=5)
        m.face_bc = np.where(m.face_bc != 0, 2, 0).astype(np.int8)
        return m
    return {"hex3": lambda: hex_mesh(3, bc=2), "prism2": lambda: prism_mesh(2, bc=2),
            "octa2": lambda: octa_mesh(2, bc=2)}[name]()


@pytest.mark.parametrize("mname", ["hex3", "prism2", "octa2", "cvt30"])
def test_k2_flux_system_and_solves(vs, mname):
    """k = 2 with flux data on the whole boundary and the mean-zero pressure:
    the eliminated saddle matrix, the right-hand side with the multiplier's
    projection and S against the oracle; MINRES and FGMRES solves against
    the oracle's direct solve of the bordered system, the multiplier value
    and int p_h = 0."""
    from oracle import assemble, solvers
    m = _flux_mesh(mname)
    K = fields.K_lognormal(m.n_cells, seed=6, sigma=0.5)
    _, u_ex, f_ex = _cubic()
    sys_ = assemble(m, paper_element(2), 1.0 / K, f=f_ex, flux=u_ex)
    assert sys_.multiplier
    tol = SYS_TOL[mname]
    s = vs.Solver(m, element=vs.VEM_ELEMENT_K2)
    try:
        s.set_coefficient(K)
        s.set_data(f_ex, None, flux=u_ex)
        A, rhs = s.system()
        S, _ = s.schur()
    finally:
        s.close()
    Ar = sys_.saddle()
    assert abs(A - Ar).max() <= tol * abs(Ar).max()
    ref = sys_.rhs()
    e, c = sys_.null_vec, sys_.cvec
    lam = (e @ ref[sys_.n_u:]) / (e @ c)
    ref[sys_.n_u:] -= c * lam
    np.testing.assert_allclose(rhs, ref, rtol=0, atol=tol * np.abs(ref).max())
    Sr = solvers.schur(sys_)
    assert abs(S - Sr).max() <= tol * abs(Sr).max()
    ud, pd, lamd = solvers.solve_direct(sys_, return_multiplier=True)
    for krylov, prec in [(0, 0), (1, 1)]:
        s = vs.Solver(m, element=vs.VEM_ELEMENT_K2, krylov=krylov, precond=prec, rtol=1e-12, inner_rtol=1e-13,
                      maxit=4000)
        try:
            s.set_coefficient(K)
            s.set_data(f_ex, None, flux=u_ex)
            u, p, st = s.solve()
        finally:
            s.close()
        assert st["relres"] <= 1e-12
        assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)
        assert np.linalg.norm(p - pd) <= 1e-9 * np.linalg.norm(pd)
        assert abs(c @ p) <= 1e-11 * np.abs(p).max() * c.sum()
        assert st["multiplier"] == pytest.approx(lamd, rel=1e-9, abs=1e-12)


def test_quadrature_points_into_device_buffer(vs):
    """The cell and boundary-face points copied into a CUDA tensor equal the
    host copy (the k = 2 cell set of a large mesh is evaluated on the
    device); a buffer of the wrong shape or type is refused."""
    import torch
    s = vs.Solver(prism_mesh(2), element=vs.VEM_ELEMENT_K2)
    try:
        for which in (vs.VEM_QP_CELL, vs.VEM_QP_BFACE):
            host = s.quadrature_points(which)
            dev = torch.full((host.shape[0], 3), np.nan, dtype=torch.float64, device="cuda")
            s.quadrature_points(which, out=dev)
            np.testing.assert_array_equal(dev.cpu().numpy(), host)
        n = s.quadrature_count(vs.VEM_QP_CELL)
        with pytest.raises(ValueError):
            s.quadrature_points(vs.VEM_QP_CELL, out=torch.empty((n, 2), dtype=torch.float64, device="cuda"))
        with pytest.raises(ValueError):
            s.quadrature_points(vs.VEM_QP_CELL, out=torch.empty((n, 3), dtype=torch.float32, device="cuda"))
    finally:
        s.close()


def test_k2_unsupported_combinations(vs):
    mesh = hex_mesh(2)
    # batched solves take the Jacobi-PCG inner solver only, as for every element
    s = vs.Solver(mesh, element=vs.VEM_ELEMENT_K2, krylov=1, precond=vs.VEM_PREC_BLOCK_TRI,
                  inner=vs.VEM_INNER_AMG)
    try:
        s.set_data(_f2, _g2)
        with pytest.raises(vs.VemError) as e:
            s.solve_batched(np.ones((2, mesh.n_cells)))
        assert e.value.code == 8
    finally:
        s.close()
    # the AMG inner solver with the multiplier pins one DOF per cell
    m = hex_mesh(2, bc=2)
    _, u_ex, f_ex = _cubic()
    s = vs.Solver(m, element=vs.VEM_ELEMENT_K2, krylov=1, precond=1, inner=vs.VEM_INNER_AMG)
    try:
        s.set_data(f_ex, None, flux=u_ex)
        with pytest.raises(vs.VemError) as e:
            s.solve()
        assert e.value.code == 8
    finally:
        s.close()
