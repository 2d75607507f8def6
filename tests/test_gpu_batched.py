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
