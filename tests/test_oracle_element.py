"""Pins for oracle/element.py: closed forms, consistency, DOF counts."""

import os

import numpy as np
import pytest

from oracle.element import E0, interpolate, local_system, paper_element
from oracle.monomials import mono3
from oracle.polyhedron import cell_geometry
from synth import affine, hex_mesh, octa_mesh, prism_mesh, tet_mesh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table_dofs.txt")
A_SHEAR = np.array([[1.0, 0.3, 0.1], [0.0, 0.8, -0.2], [0.1, 0.0, 1.2]])


def _cells():
    yield "cube", cell_geometry(hex_mesh(1), 0)
    yield "sheared", cell_geometry(affine(hex_mesh(1), A_SHEAR, (0.3, 0.1, -0.2)), 0)
    yield "tet", cell_geometry(tet_mesh(1), 2)
    yield "prism", cell_geometry(prism_mesh(1), 1)


def _mesh_counts(kind, n):
    """(faces, cells): Cube n^3 has 3n^2(n+1) faces; Octa (9 cells per cube)
    has 20 n^3 + 12 n^2 (n+1) (8 octahedron faces and 12 mid-plane triangles
    inside each cube, 4 quarter squares on each cube face)."""
    if kind == "cube":
        return 3 * n * n * (n + 1), n ** 3
    return 20 * n ** 3 + 12 * n * n * (n + 1), 9 * n ** 3


def test_dof_counts_match_paper_tables():
    """Total = face DOFs + interior DOFs + pressure DOFs, and the paper's
    tables print that total + 1 (the mean-zero pressure multiplier of its
    Neumann problem, Sec. 3).  The Octa rows fix the Octa family's cell and
    face counts, from which synth.octa_mesh was built."""
    rows = [l.split() for l in open(GOLDEN) if l.strip() and not l.startswith("#")]
    assert len(rows) == 16
    for r in rows:
        n, k, dofs = int(r[1]), int(r[2]), int(r[3])
        spec = paper_element(k)
        F, Nc = _mesh_counts(r[0], n)
        total = spec.nfd * F + (spec.nid + spec.nq) * Nc
        assert total + 1 == dofs, r


@pytest.mark.parametrize("n", [1, 2, 4])
def test_octa_mesh_counts_and_cells(n):
    """The generated Octa mesh has the counts above, cells of seven or eight
    faces, and cell volumes h^3/6 (octahedron on the face centres of a cube
    of side h) and (h^3 - h^3/6)/8 = 5h^3/48 (corner pieces), summing to 1."""
    m = octa_mesh(n)
    F, Nc = _mesh_counts("octa", n)
    assert (m.n_faces, m.n_cells) == (F, Nc)
    nfc = np.diff(m.cell_face_ptr)
    assert np.array_equal(np.bincount(nfc, minlength=9)[7:], [8 * n ** 3, n ** 3])
    h = 1.0 / n
    vols = np.array([cell_geometry(m, c).volume for c in range(m.n_cells)])
    np.testing.assert_allclose(vols[nfc == 8], h ** 3 / 6, rtol=1e-13)
    np.testing.assert_allclose(vols[nfc == 7], 5 * h ** 3 / 48, rtol=1e-13)
    assert vols.sum() == pytest.approx(1.0, rel=1e-13)


def test_octa_table_dofs_from_generated_mesh():
    """Table 5's N_P = 576 row (k = 2: 23809 DOFs) counted on the generated
    mesh itself."""
    m = octa_mesh(4)
    spec = paper_element(2)
    assert m.n_cells == 576
    assert spec.nfd * m.n_faces + (spec.nid + spec.nq) * m.n_cells + 1 == 23809


@pytest.mark.parametrize("spec", [E0, paper_element(1), paper_element(2)], ids=lambda s: s.name)
def test_local_matrix_symmetric_spd_and_projector(spec):
    for name, cell in _cells():
        loc = local_system(cell, spec, 1.7, details=True)
        M = loc["M"]
        np.testing.assert_allclose(M, M.T, atol=1e-13 * np.abs(M).max())
        assert np.linalg.eigvalsh(M).min() > 0, name
        # [P_kp]^3 is inside the local space: Pi D = I
        np.testing.assert_allclose(loc["Pi"] @ loc["D"], np.eye(loc["D"].shape[1]), atol=1e-11)


@pytest.mark.parametrize("spec", [E0, paper_element(1), paper_element(2)], ids=lambda s: s.name)
def test_consistency_on_polynomials(spec):
    """For v in [P_kp]^3 the discrete form is exact: I(v)^T M_P I(w) = nu int v.w,
    and B_P I(v) = int div v psi (div v in P_kq), with I the DOF interpolant."""
    rng = np.random.default_rng(7)
    nu = 2.3
    for name, cell in _cells():
        loc = local_system(cell, spec, nu, details=True)
        pal = mono3(spec.kp)
        cv = rng.standard_normal((2, 3, len(pal)))

        def field(cf):
            def v(X):
                Y = (X - cell.centroid) / cell.diameter
                out = np.zeros((X.shape[0], 3))
                for c in range(3):
                    for j, a in enumerate(pal):
                        out[:, c] += cf[c, j] * Y[:, 0] ** a[0] * Y[:, 1] ** a[1] * Y[:, 2] ** a[2]
                return out
            return v
        v, w = field(cv[0]), field(cv[1])
        Iv, Iw = interpolate(cell, spec, v), interpolate(cell, spec, w)
        exact = nu * np.sum(cell.qw * np.sum(v(cell.qp) * w(cell.qp), 1))
        assert Iv @ loc["M"] @ Iw == pytest.approx(exact, rel=1e-10), name
        if spec.kq == 0:
            # int_P div v = int_dP v.n (divergence theorem)
            flux = sum(F.sigma * np.sum(F.qw * (v(F.qp) @ F.normal)) for F in cell.faces)
            assert (loc["B"] @ Iv)[0] == pytest.approx(flux, rel=1e-10, abs=1e-12), name


def test_E0_cube_closed_form():
    """E0 on a cube of side a, global normals along +axes: per axis the two
    opposite faces couple as nu a^3 [[3/4, -1/4], [-1/4, 3/4]] (consistency
    nu/|P| N N^T plus stabilisation nu |P| (I - D Pi)^T (I - D Pi), worked out
    by hand), different axes do not couple, and B_P = sigma |f|."""
    a, nu = 0.5, 3.0
    m = affine(hex_mesh(1), a * np.eye(3), (0.1, 0.2, 0.3))
    cell = cell_geometry(m, 0)
    loc = local_system(cell, E0, nu)
    ref = np.zeros((6, 6))
    for ax in range(3):
        i, j = 2 * ax, 2 * ax + 1
        ref[i, i] = ref[j, j] = 0.75
        ref[i, j] = ref[j, i] = -0.25
    np.testing.assert_allclose(loc["M"], nu * a ** 3 * ref, atol=1e-14)
    np.testing.assert_allclose(loc["B"][0], a * a * np.array([-1, 1, -1, 1, -1, 1]), atol=1e-15)


@pytest.mark.parametrize("spec", [E0, paper_element(1)], ids=lambda s: s.name)
def test_scaling(spec):
    """M_P scales as nu h^3 under x -> s x (DOFs are scale-free, eq. facePoly-
    crossMom); B_P scales as h^2."""
    c1 = cell_geometry(affine(hex_mesh(1), A_SHEAR), 0)
    c2 = cell_geometry(affine(hex_mesh(1), 0.25 * A_SHEAR), 0)
    l1 = local_system(c1, spec, 1.0)
    l2 = local_system(c2, spec, 5.0)
    np.testing.assert_allclose(l2["M"], 5.0 * 0.25 ** 3 * l1["M"], rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(l2["B"], 0.25 ** 2 * l1["B"], rtol=1e-10, atol=1e-14)


def test_stabilisation_vanishes_on_polynomials():
    """s_P(v - Pi v, .) = 0 for v in [P_k]^3: (I - D Pi) D = 0."""
    for name, cell in _cells():
        loc = local_system(cell, paper_element(1), 1.0, details=True)
        R = np.eye(loc["D"].shape[0]) - loc["D"] @ loc["Pi"]
        np.testing.assert_allclose(R @ loc["D"], 0, atol=1e-11)
