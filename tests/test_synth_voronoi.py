"""Pins for the seeded Voronoi / CVT mesh generator (an input generator):
closed cells, volumes that tile the cube, and the bisector property of
interior faces."""

import numpy as np
import pytest

from synth.voronoi import voronoi_mesh


@pytest.mark.parametrize("n,lloyd", [(40, 0), (300, 5)])
def test_voronoi_mesh_is_a_tiling(n, lloyd):
    mesh, seeds = voronoi_mesh(n, seed=4, lloyd=lloyd, return_seeds=True)
    mesh.validate()
    assert mesh.n_cells == n
    # face area vectors (Newell) and the orientation of each face in each cell
    fvec = np.zeros((mesh.n_faces, 3))
    for f in range(mesh.n_faces):
        V = mesh.xyz[mesh.face_vertices(f)]
        fvec[f] = 0.5 * np.cross(V, np.roll(V, -1, 0)).sum(0)
    owner = -np.ones(mesh.n_faces, dtype=int)
    vol = np.zeros(n)
    for c in range(n):
        s = np.zeros(3)
        for f in mesh.cell_faces(c):
            V = mesh.xyz[mesh.face_vertices(f)]
            ctr = V.mean(0)
            out = 1.0 if np.dot(ctr - seeds[c], fvec[f]) > 0 else -1.0
            s += out * fvec[f]
            vol[c] += out * np.dot(ctr, fvec[f]) / 3.0   # divergence theorem
            if owner[f] < 0:
                owner[f] = c
        assert np.linalg.norm(s) < 1e-12, "open cell"
    assert vol.sum() == pytest.approx(1.0, rel=1e-12)
    assert np.all(vol > 0)
    # interior faces lie on the bisector of their two seeds, oriented i -> j
    cells_of = [[] for _ in range(mesh.n_faces)]
    for c in range(n):
        for f in mesh.cell_faces(c):
            cells_of[f].append(c)
    for f in range(mesh.n_faces):
        if len(cells_of[f]) == 2:
            i, j = sorted(cells_of[f])
            V = mesh.xyz[mesh.face_vertices(f)]
            di = np.linalg.norm(V - seeds[i], axis=1)
            dj = np.linalg.norm(V - seeds[j], axis=1)
            np.testing.assert_allclose(di, dj, atol=1e-10)
            assert np.dot(fvec[f], seeds[j] - seeds[i]) > 0


def test_cvt_face_statistics():
    """Lloyd-relaxed meshes have ~13-15 faces per cell (the paper's CVT tables
    imply about 13.3-13.5 interior faces per cell)."""
    mesh = voronoi_mesh(2000, seed=0, lloyd=10)
    nf = np.diff(mesh.cell_face_ptr)
    assert 13.0 < nf.mean() < 15.0
