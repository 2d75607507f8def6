"""Optimality of the Block-Schur preconditioner under refinement (the
paper's optimality test, Sec. 5, here at k = 1 and with the paper's flux
boundary data and mean-zero pressure): with S solved to 1e-12 the FGMRES
iteration count stays bounded as the Cube, Octa and CVT meshes are
refined."""

import numpy as np
import pytest

from synth import fields, hex_mesh, octa_mesh
from synth.voronoi import voronoi_mesh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    return vemsolve


def _iters(vs, mesh):
    prob = fields.paper_polynomial_problem()
    s = vs.Solver(mesh, element=1, krylov=1, precond=0, restart=30, rtol=1e-8, inner=vs.VEM_INNER_AMG,
                  inner_rtol=1e-12, maxit=3000)
    try:
        s.set_data(prob.f, prob.gD, flux=prob.u)
        _, _, st = s.solve()
    finally:
        s.close()
    assert st["relres"] <= 1e-8
    return st["iterations"]


def _neumann(m):
    m.face_bc = np.where(m.face_bc != 0, 2, 0).astype(np.int8)
    return m


def _mesh(family, n):
    if family == "cube":
        return hex_mesh(n, bc=2)
    if family == "octa":
        return octa_mesh(n, bc=2)
    return _neumann(voronoi_mesh(n, seed=7, lloyd=10))


@pytest.mark.parametrize("family,sizes", [("cube", (8, 16, 24)), ("octa", (2, 4, 8)),
                                          ("cvt", (1000, 4000, 8000))])
def test_block_schur_iterations_bounded(vs, family, sizes):
    its = []
    for n in sizes:
        m = _mesh(family, n)
        its.append(_iters(vs, m))
    for a, b in zip(its, its[1:]):
        assert b <= 1.1 * a + 2, its
