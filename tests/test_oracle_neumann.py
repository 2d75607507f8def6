"""Pins for prescribed-flux (Neumann) faces and the mean-zero pressure of
the paper's model problem (Sec. 3: u.n = u_N on the boundary, pressure in
Q = {int q = 0}, one Lagrange multiplier)."""

import numpy as np
import scipy.sparse as sp
import pytest

from oracle import E0, assemble, paper_element, solvers
from oracle.assemble import mesh_cells
from oracle.element import interpolate
from synth import affine, fields, hex_mesh, octa_mesh, prism_mesh, tet_mesh
from synth.voronoi import voronoi_mesh

A_SHEAR = np.array([[1.0, 0.3, 0.1], [0.0, 0.8, -0.2], [0.1, 0.0, 1.2]])
MESHES = {
    "hex": lambda bc: hex_mesh(3, bc=bc),
    "tet": lambda bc: tet_mesh(2, bc=bc),
    "prism": lambda bc: prism_mesh(2, bc=bc),
    "octa": lambda bc: octa_mesh(1, bc=bc),
    "voronoi": lambda bc: _with_bc(voronoi_mesh(30, seed=3, lloyd=2), bc),
}


def _with_bc(m, bc):
    m.face_bc = np.where(m.face_bc != 0, bc, 0).astype(np.int8)
    return m


def _mixed_bc(m):
    """Dirichlet on the faces whose centroid has x < 1e-9, flux elsewhere."""
    fb = m.face_bc.copy()
    for f in np.nonzero(fb)[0]:
        xs = m.xyz[m.face_vertices(f)]
        fb[f] = 1 if np.all(np.abs(xs[:, 0]) < 1e-9) else 2
    m.face_bc = fb.astype(np.int8)
    return m


def _interp(sys, spec, cells, mesh, v):
    from oracle.assemble import cell_dofmap
    uI = np.zeros(sys.n_u)
    for c, cell in enumerate(cells):
        uI[cell_dofmap(mesh, c, spec)] = interpolate(cell, spec, v)
    return uI


@pytest.mark.parametrize("mesh", list(MESHES))
@pytest.mark.parametrize("spec,probname", [(E0, "linear"), (paper_element(1), "linear"),
                                           (paper_element(1), "quadratic")],
                         ids=["E0-lin", "E1-lin", "E1-quad"])
def test_neumann_patch(mesh, spec, probname):
    """All-flux boundary, constant K, p in P_{kp+1}: u_h is the interpolant
    of the exact flux and p_h the cell means of p minus their volume-weighted
    mean (the mean-zero member of the solution family)."""
    m = MESHES[mesh](2)
    K = 2.5
    prob = fields.linear_problem(K=K) if probname == "linear" else fields.quadratic_problem(K=K)
    sys = assemble(m, spec, np.full(m.n_cells, 1.0 / K), f=prob.f, flux=prob.u)
    assert sys.multiplier and sys.fixed.size == spec.nfd * int((m.face_bc == 2).sum())
    u, p, lam = solvers.solve_direct(sys, return_multiplier=True)
    cells = mesh_cells(m)
    uI = _interp(sys, spec, cells, m, prob.u)
    pI = np.array([(cell.qw @ prob.p(cell.qp)) / cell.volume for cell in cells])
    pI -= sys.vol @ pI / sys.vol.sum()
    np.testing.assert_allclose(u, uI, atol=1e-10 * max(1, np.abs(uI).max()))
    np.testing.assert_allclose(p, pI, atol=1e-10)
    assert abs(sys.vol @ p) <= 1e-12
    assert abs(lam) <= 1e-10          # compatible data: the multiplier vanishes


def test_multiplier_is_mean_of_incompatible_source():
    """f = 1 with zero boundary flux has no solution in the plain sense; the
    multiplier absorbs the mean of f (lambda = int f / |Omega| = 1)."""
    m = hex_mesh(3, bc=2)
    sys = assemble(m, E0, np.ones(m.n_cells), f=lambda x: np.ones(x.shape[0]),
                   flux=lambda x: np.zeros_like(x))
    u, p, lam = solvers.solve_direct(sys, return_multiplier=True)
    assert lam == pytest.approx(1.0, rel=1e-12)
    np.testing.assert_allclose(u, 0.0, atol=1e-12)


@pytest.mark.parametrize("spec", [E0, paper_element(1)], ids=lambda s: s.name)
def test_mixed_boundary_patch(spec):
    """Dirichlet on x = 0, flux elsewhere: no multiplier, exact for linear p."""
    m = affine(_mixed_bc(hex_mesh(2)), A_SHEAR, (0.0, 0.0, 0.0))
    prob = fields.linear_problem(K=1.0)
    sys = assemble(m, spec, np.ones(m.n_cells), f=prob.f, gD=prob.gD, flux=prob.u)
    assert not sys.multiplier
    u, p = solvers.solve_direct(sys)
    cells = mesh_cells(m)
    uI = _interp(sys, spec, cells, m, prob.u)
    pI = np.array([(cell.qw @ prob.p(cell.qp)) / cell.volume for cell in cells])
    np.testing.assert_allclose(u, uI, atol=1e-10 * max(1, np.abs(uI).max()))
    np.testing.assert_allclose(p, pI, atol=1e-10)


@pytest.mark.parametrize("mesh", ["sheared", "prism"])
def test_mixed_boundary_patch_k2(mesh):
    """k = 2, pressure data on x = 0 and flux data elsewhere, constant K and
    p in P_3 (flux in [P_2]^3): no multiplier, u_h is the interpolant and
    p_h the P_1 moments of p.  The boundary data rule of k = 2 (degree 5)
    integrates g_D m^f and (u.n) m^f exactly."""
    from oracle.monomials import eval_mono3, mono3
    spec = paper_element(2)
    base = hex_mesh(2) if mesh == "sheared" else prism_mesh(2)
    m = _mixed_bc(base)
    if mesh == "sheared":
        A = np.array([[1.0, 0.0, 0.0], [0.3, 0.8, -0.2], [0.1, 0.0, 1.2]])
        m = affine(m, A, (0.0, 0.0, 0.0))
    K = 1.3
    p_ex, u_ex, f_ex = _cubic_problem(K)
    sys = assemble(m, spec, np.full(m.n_cells, 1.0 / K), f=f_ex, gD=p_ex, flux=u_ex)
    assert not sys.multiplier and sys.fixed.size > 0
    u, p = solvers.solve_direct(sys)
    cells = mesh_cells(m)
    uI = _interp(sys, spec, cells, m, u_ex)
    pI = np.concatenate([(cell.qw * p_ex(cell.qp)) @ eval_mono3(mono3(1), cell.qp, cell.centroid, cell.diameter)
                         / cell.volume for cell in cells])
    np.testing.assert_allclose(u, uI, atol=1e-10 * max(1, np.abs(uI).max()))
    np.testing.assert_allclose(p, pI, atol=1e-10 * max(1, np.abs(pI).max()))


@pytest.mark.parametrize("spec", [E0, paper_element(1)], ids=lambda s: s.name)
def test_neumann_conservation_and_krylov(spec):
    """Paper's polynomial solution with flux data: B u_h = F - c lambda per
    cell (local conservation up to the multiplier), and the Block-Schur
    Krylov solves (exact S on the augmented Schur block, or AMG-PCG) reach the
    direct solution."""
    m = prism_mesh(2, bc=2)
    prob = fields.paper_polynomial_problem()
    nu = 1.0 / fields.K_lognormal(m.n_cells, seed=4, sigma=0.5)
    sys = assemble(m, spec, nu, f=prob.f, flux=prob.u)
    u, p, lam = solvers.solve_direct(sys, return_multiplier=True)
    keep = np.ones(sys.n_u)
    keep[sys.fixed] = 0.0
    r = sys.rhs()[sys.n_u:] - sys.vol * lam
    np.testing.assert_allclose(sys.B @ (u * keep), r, atol=1e-10 * np.abs(r).max())
    for method, kind, inner in [("fgmres", "diag", "exact"), ("fgmres", "tri", "amg"), ("minres", "diag", "exact")]:
        uk, pk, res = solvers.solve_krylov(sys, method, kind, inner, rtol=1e-11, inner_rtol=1e-13)
        assert res.converged
        np.testing.assert_allclose(uk, u, atol=1e-8 * np.abs(u).max())
        np.testing.assert_allclose(pk, p, atol=1e-8 * np.abs(p).max())


def _cubic_problem(K):
    """p in P_3, constant K: u = -K grad p in [P_2]^3, f = div u in P_1."""
    def p(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return X ** 3 - 2 * X * Y * Y + 0.5 * Z ** 3 + X * Y * Z + Y * Y - 0.4 * Z

    def u(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return -K * np.stack([3 * X * X - 2 * Y * Y + Y * Z, -4 * X * Y + X * Z + 2 * Y,
                              1.5 * Z * Z + X * Y - 0.4], 1)

    def f(x):
        X, Y, Z = x[:, 0], x[:, 1], x[:, 2]
        return -K * (6 * X - 4 * X + 2 + 3 * Z)

    return p, u, f


@pytest.mark.parametrize("mesh", ["hex", "prism", "octa", "voronoi"])
def test_neumann_patch_k2(mesh):
    """The k = 2 element with flux data on the whole boundary, constant K and
    p in P_3: u_h is the interpolant of the exact flux, the pressure DOFs
    are the P_1 moments (1/|P|) int_P p m_q shifted along the constants to
    int p_h = 0, and the multiplier vanishes (compatible data)."""
    from oracle.monomials import eval_mono3, mono3
    spec = paper_element(2)
    m = MESHES[mesh](2)
    K = 1.7
    p_ex, u_ex, f_ex = _cubic_problem(K)
    sys = assemble(m, spec, np.full(m.n_cells, 1.0 / K), f=f_ex, flux=u_ex)
    assert sys.multiplier and sys.n_p == 4 * m.n_cells
    u, p, lam = solvers.solve_direct(sys, return_multiplier=True)
    cells = mesh_cells(m)
    uI = _interp(sys, spec, cells, m, u_ex)
    pI = np.concatenate([(cell.qw * p_ex(cell.qp)) @ eval_mono3(mono3(1), cell.qp, cell.centroid, cell.diameter)
                         / cell.volume for cell in cells])
    e, c = sys.null_vec, sys.cvec
    pI -= (c @ pI) / (c @ e) * e
    np.testing.assert_allclose(u, uI, atol=1e-9 * max(1, np.abs(uI).max()))
    np.testing.assert_allclose(p, pI, atol=1e-9 * max(1, np.abs(pI).max()))
    assert abs(c @ p) <= 1e-12 * np.abs(p).max()
    assert abs(lam) <= 1e-9


def test_neumann_k2_multiplier_and_krylov():
    """k = 2, the paper's polynomial solution with flux data: local
    conservation up to the multiplier (B u_h = F - c lambda), the kernel of
    B^T is the constant moments, and Block-Schur Krylov solves with the exact
    bordered Schur block reach the direct solution."""
    spec = paper_element(2)
    m = hex_mesh(2, bc=2)
    prob = fields.paper_polynomial_problem()
    sys = assemble(m, spec, 1.0 / fields.K_lognormal(m.n_cells, seed=4, sigma=0.5), f=prob.f, flux=prob.u)
    u, p, lam = solvers.solve_direct(sys, return_multiplier=True)
    keep = np.ones(sys.n_u)
    keep[sys.fixed] = 0.0
    Bk = sys.B @ sp.diags(keep)
    np.testing.assert_allclose(Bk.T @ sys.null_vec, 0.0, atol=1e-12 * abs(sys.B).max())
    r = sys.rhs()[sys.n_u:] - sys.cvec * lam
    np.testing.assert_allclose(Bk @ u, r, atol=1e-10 * np.abs(r).max())
    for method, kind in [("fgmres", "diag"), ("fgmres", "tri"), ("minres", "diag")]:
        uk, pk, res = solvers.solve_krylov(sys, method, kind, "exact", rtol=1e-11)
        assert res.converged
        np.testing.assert_allclose(uk, u, atol=1e-8 * np.abs(u).max())
        np.testing.assert_allclose(pk, p, atol=1e-8 * np.abs(p).max())
