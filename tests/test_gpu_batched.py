"""Batched solves (vem_solve_batched): systems on one mesh with their own K
and source, as one stacked launch sequence; every system matches its own
single solve and the oracle."""

import numpy as np
import pytest

from oracle import E0, assemble, paper_element, solvers
from synth import fields, hex_mesh, prism_mesh
from synth.voronoi import voronoi_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    return vemsolve


@pytest.mark.parametrize("case", ["E0-hex", "K1-prism", "E0-cvt"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batched_matches_oracle(vs, case, precision):
    mk, spec, elem = {"E0-hex": (lambda: hex_mesh(4), E0, 0),
                      "K1-prism": (lambda: prism_mesh(3), paper_element(1), 1),
                      "E0-cvt": (lambda: voronoi_mesh(50, seed=1, lloyd=3), E0, 0)}[case]
    mesh = mk()
    nb = 5
    Ks = np.stack([fields.K_lognormal(mesh.n_cells, seed=100 + b, sigma=2.0) for b in range(nb)])
    srcs = [fields.fourier_source(200 + b) for b in range(nb)]
    s = vs.Solver(mesh, element=elem, krylov=1, precond=1, precision=precision, rtol=1e-11,
                  inner_rtol=1e-12 if precision == 0 else 1e-5, maxit=3000)
    xc = s.quadrature_points(vs.VEM_QP_CELL)
    F = np.stack([src(xc) for src in srcs])
    U, P, rel, st = s.solve_batched(Ks, F, None)
    assert np.all(rel <= 1e-11), rel
    for b in range(nb):
        sys = assemble(mesh, spec, 1.0 / Ks[b], f=srcs[b])
        ud, pd = solvers.solve_direct(sys)
        assert np.linalg.norm(U[b] - ud) <= 1e-8 * np.linalg.norm(ud), b
        assert np.linalg.norm(P[b] - pd) <= 1e-8 * np.linalg.norm(pd), b
    # a single solve afterwards still works (the batched call invalidated the assembly)
    s.set_coefficient(Ks[2])
    s.set_source(F[2], None)
    u, p, st1 = s.solve()
    assert np.linalg.norm(u - U[2]) <= 1e-8 * np.linalg.norm(U[2])
    s.close()


def _quad_f(c):
    def f(x):
        return c[0] + x @ c[1:4] + c[4] * x[:, 0] * x[:, 2] - c[5] * x[:, 1] ** 2
    return f


@pytest.mark.parametrize("case", ["hex3", "prism2"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batched_k2_matches_oracle(vs, case, precision):
    """The paper's k = 2 element in a batch: per-system coefficients, loads at
    the fan-tetrahedron cell points and Dirichlet data, the block-triangular
    flux update from the copied B^T rows of every system, per-system FGMRES
    and inner Jacobi-PCG on the 4 x 4-block Schur matrices.  Data of degree
    <= 2, for which the library's and the oracle's load rules are both
    exact; every system matches the oracle's direct solve and its own single
    solve."""
    mesh = {"hex3": lambda: hex_mesh(3), "prism2": lambda: prism_mesh(2)}[case]()
    K2 = paper_element(2)
    nb = 4
    rng = np.random.default_rng(71)
    Ks = np.stack([fields.K_lognormal(mesh.n_cells, seed=300 + b, sigma=1.0) for b in range(nb)])
    fs = [_quad_f(rng.standard_normal(6)) for _ in range(nb)]
    gs = [_quad_f(rng.standard_normal(6)) for _ in range(nb)]
    s = vs.Solver(mesh, element=vs.VEM_ELEMENT_K2, krylov=1, precond=1, precision=precision, rtol=1e-11,
                  inner_rtol=1e-12 if precision == 0 else 1e-5, maxit=3000)
    try:
        xc = s.quadrature_points(vs.VEM_QP_CELL)
        xb = s.quadrature_points(vs.VEM_QP_BFACE)
        F = np.stack([f(xc) for f in fs])
        G = np.stack([g(xb) for g in gs])
        with pytest.raises(ValueError):
            s.solve_batched(Ks, F[:, :-1], G)
        U, P, rel, st = s.solve_batched(Ks, F, G)
        assert np.all(rel <= 1e-11), rel
        assert U.shape == (nb, st["n_u"] // nb) and P.shape == (nb, 4 * mesh.n_cells)
        for b in range(nb):
            sys_ = assemble(mesh, K2, 1.0 / Ks[b], f=fs[b], gD=gs[b])
            ud, pd = solvers.solve_direct(sys_)
            assert np.linalg.norm(U[b] - ud) <= 1e-8 * np.linalg.norm(ud), b
            assert np.linalg.norm(P[b] - pd) <= 1e-8 * np.linalg.norm(pd), b
        s.set_coefficient(Ks[1])
        s.set_source(F[1], G[1])
        u, p, _ = s.solve()
        assert np.linalg.norm(u - U[1]) <= 1e-8 * np.linalg.norm(U[1])
        assert np.linalg.norm(p - P[1]) <= 1e-8 * np.linalg.norm(P[1])
    finally:
        s.close()


def test_batched_rejects_bad_K(vs):
    s = vs.Solver(hex_mesh(2))
    K = np.ones((3, 8))
    K[1, 4] = 0.0
    with pytest.raises(vs.VemError) as e:
        s.solve_batched(K)
    assert e.value.code == 1


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batched_systems_are_independent(vs, precision):
    """Every system of a batch runs its own FGMRES and its own inner PCG
    (own scalars, own stopping test): with the batch size and position fixed,
    a system's solution does not depend, bit for bit, on the other systems,
    and a system with zero data stops at once while the others iterate."""
    mesh = hex_mesh(5)
    nc = mesh.n_cells
    K = [fields.K_lognormal(nc, seed=300 + b, sigma=2.0) for b in range(3)]
    s = vs.Solver(mesh, element=0, krylov=1, precond=1, precision=precision, rtol=1e-10,
                  inner_rtol=1e-8 if precision == 0 else 1e-5, maxit=3000)
    xc = s.quadrature_points(vs.VEM_QP_CELL)
    F0 = fields.fourier_source(400)(xc)
    F1 = fields.fourier_source(401)(xc)
    try:
        Ua, Pa, ra, _ = s.solve_batched(np.stack([K[0], K[1]]), np.stack([F0, F1]), None)
        Ub, Pb, rb, _ = s.solve_batched(np.stack([K[0], K[2]]), np.stack([F0, 3.0 * F1]), None)
        Uc, Pc, rc, _ = s.solve_batched(np.stack([K[0], K[1]]), np.stack([F0, np.zeros(nc)]), None)
    finally:
        s.close()
    np.testing.assert_array_equal(Ua[0], Ub[0])
    np.testing.assert_array_equal(Pa[0], Pb[0])
    np.testing.assert_array_equal(Ua[0], Uc[0])
    assert np.all(Uc[1] == 0.0) and np.all(Pc[1] == 0.0)
    assert ra[0] <= 1e-10 and rb[1] <= 1e-10
