"""Pins for oracle/schwarz.py: edge patches, the additive Schwarz operator,
its Lanczos spectral estimate and Block-Reg at the paper's k = 2 with the
edge-patch smoother on the finest level of the A_reg AMG."""

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import E0, assemble, paper_element, schwarz, solvers
from synth import fields, hex_mesh
from synth.voronoi import voronoi_mesh

K1, K2 = paper_element(1), paper_element(2)


def _areg(m, spec, **kw):
    sys_ = assemble(m, spec, np.ones(m.n_cells), **kw)
    return sys_, solvers.regularized(sys_, solvers.mesh_size(sys_) ** 2).tocsr()


def test_edge_patches_on_cubes():
    """n^3 cubes: 3 n (n+1)^2 edges; a patch holds the faces around its edge
    (4 inside the cube, 3 on a side, 2 on an edge of the cube) and the cells
    touching them (4, 2, 1); every quad face lies in 4 patches (its edges)
    and every cell's interior DOFs in 12 (the edges of a hexahedron)."""
    n = 3
    m = hex_mesh(n)
    P = schwarz.edge_patches(m, K1)
    assert len(P) == 3 * n * (n + 1) ** 2
    sizes = sorted({p.size for p in P})
    assert sizes == [2 * 3 + 1 * 3, 3 * 3 + 2 * 3, 4 * 3 + 4 * 3]
    count = np.zeros(K1.nfd * m.n_faces + K1.nid * m.n_cells, dtype=int)
    for p in P:
        assert np.all(np.diff(p) > 0)
        count[p] += 1
    assert np.all(count[:K1.nfd * m.n_faces] == 4)
    assert np.all(count[K1.nfd * m.n_faces:] == 12)


def test_schwarz_operator_special_cases():
    """One patch holding every DOF gives M_S = A^-1; patches that partition
    the DOFs give the block-Jacobi inverse."""
    _, A = _areg(hex_mesh(2), K1)
    n = A.shape[0]
    M1 = schwarz.schwarz_operator(A, [np.arange(n)]).toarray()
    np.testing.assert_allclose(M1, np.linalg.inv(A.toarray()), rtol=0, atol=1e-12 * np.abs(M1).max())
    parts = np.array_split(np.arange(n), 7)
    M2 = schwarz.schwarz_operator(A, parts).toarray()
    ref = np.zeros((n, n))
    Ad = A.toarray()
    for G in parts:
        ref[np.ix_(G, G)] = np.linalg.inv(Ad[np.ix_(G, G)])
    np.testing.assert_allclose(M2, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("spec", [K1, K2], ids=["K1", "K2"])
def test_lanczos_estimate_of_the_schwarz_spectrum(spec):
    """M_S A is self-adjoint in the A-inner product with positive spectrum;
    the A-Lanczos Ritz value lies below its largest eigenvalue and within
    10% of it after 10 steps."""
    m = hex_mesh(2)
    _, A = _areg(m, spec)
    MS = schwarz.schwarz_operator(A, schwarz.edge_patches(m, spec))
    Ad = A.toarray()
    lam = np.linalg.eigvals(MS.toarray() @ Ad)
    assert np.abs(lam.imag).max() <= 1e-9 * np.abs(lam.real).max()
    lam = lam.real
    assert lam.min() > 0.0
    theta = schwarz.lanczos_max_A(A, MS)
    assert theta <= lam.max() * (1 + 1e-10)
    assert theta >= 0.9 * lam.max()


def test_cycle_symmetric_positive_definite():
    m = hex_mesh(3)
    _, A = _areg(m, K2)
    cyc = schwarz.setup(A, schwarz.edge_patches(m, K2), coarse_max=16)
    assert len(cyc.H.levels) >= 2
    n = A.shape[0]
    C = np.column_stack([cyc(e) for e in np.eye(n)])
    np.testing.assert_allclose(C, C.T, atol=1e-12 * np.abs(C).max())
    assert np.linalg.eigvalsh(0.5 * (C + C.T)).min() > 0.0


@pytest.mark.parametrize("case", ["k2-dirichlet", "k2-flux", "k1-voronoi", "e0-voronoi"])
def test_block_reg_with_edge_patches_reaches_direct_solution(case):
    prob = fields.paper_polynomial_problem()
    if case.startswith("k2"):
        flux = case.endswith("flux")
        m = hex_mesh(3, bc=2 if flux else 1)
        spec = K2
    else:
        flux = False
        m = voronoi_mesh(40, seed=3, lloyd=3)
        spec = K1 if case.startswith("k1") else E0
    kw = dict(f=prob.f, flux=prob.u) if flux else dict(f=prob.f, gD=prob.gD)
    sys_ = assemble(m, spec, np.ones(m.n_cells), **kw)
    ud, pd = solvers.solve_direct(sys_)
    u, p, res = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-11, restart=30, maxit=3000,
                                     reg_smoother="edge-schwarz", mesh=m)
    assert res.converged
    np.testing.assert_allclose(u, ud, atol=1e-8 * np.abs(ud).max())
    np.testing.assert_allclose(p, pd, atol=1e-8 * np.abs(pd).max())


def test_edge_patches_make_k2_block_reg_converge():
    """k = 2 on 3^3 cubes: with the Chebyshev point smoother the A_reg cycle
    barely reduces the error and Block-Reg FGMRES(30) does not reach 1e-8 in
    400 iterations; with the edge-patch smoother it does in under 100."""
    prob = fields.paper_polynomial_problem()
    m = hex_mesh(3)
    sys_ = assemble(m, K2, np.ones(m.n_cells), f=prob.f, gD=prob.gD)
    _, _, r_cheb = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-8, restart=30, maxit=400)
    _, _, r_edge = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-8, restart=30, maxit=400,
                                        reg_smoother="edge-schwarz", mesh=m)
    assert not r_cheb.converged
    assert r_edge.converged and r_edge.iters < 100, r_edge.iters
