"""Parity of the paper's k = 2 element matrices (Sec. 4.1-4.3 at k = 2: six
face moments, three gradient and eleven cross moments, P1 pressure) between
the CUDA element kernel and the oracle's local system, cell by cell, on hex,
sheared hex, tet, prism, Octa and Voronoi meshes; and the status of the
global paths, which are not built for k = 2."""

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


def test_k2_global_paths_unsupported(vs):
    mesh = hex_mesh(2)
    s = vs.Solver(mesh, element=vs.VEM_ELEMENT_K2)
    try:
        with pytest.raises(vs.VemError) as e:
            s.solve()
        assert e.value.code == 8
        with pytest.raises(vs.VemError) as e:
            s.assemble()
        assert e.value.code == 8
        # switching to k = 1 on the same handle assembles and solves
        s.set_options(element=vs.VEM_ELEMENT_K1)
        prob = fields.sine_problem()
        s.set_data(prob.f, prob.gD)
        _, _, st = s.solve()
        assert st["relres"] <= 1e-10
    finally:
        s.close()
