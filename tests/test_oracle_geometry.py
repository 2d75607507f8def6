"""Pins for oracle/quadrature.py and oracle/polyhedron.py against closed forms."""

from math import factorial

import numpy as np
import pytest

from oracle.polyhedron import cell_geometry, face_geometry
from oracle.quadrature import dunavant4, radon5, tet_rule, triangle_rule
from synth import affine, hex_mesh, tet_mesh


def _bary_integral(a, b, c, area):
    # int_T l1^a l2^b l3^c = 2|T| a! b! c! / (a+b+c+2)!
    return 2 * area * factorial(a) * factorial(b) * factorial(c) / factorial(a + b + c + 2)


@pytest.mark.parametrize("rule", ["gauss", "dunavant", "radon"])
def test_triangle_rules_exact(rule):
    rng = np.random.default_rng(0)
    A, B, C = rng.uniform(-1, 1, (3, 3))
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
    if rule == "gauss":
        pts, w = triangle_rule(A, B, C, 5)
        maxdeg, tol = 8, 1e-13
    elif rule == "dunavant":
        pts, w = dunavant4(A, B, C)
        maxdeg, tol = 4, 1e-13
    else:
        pts, w = radon5(A, B, C)
        maxdeg, tol = 5, 1e-13
    # barycentric coordinates of the points
    T = np.stack([B - A, C - A], 1)
    lam = np.linalg.lstsq(T, (pts - A).T, rcond=None)[0].T
    l2, l3 = lam[:, 0], lam[:, 1]
    l1 = 1 - l2 - l3
    for a in range(maxdeg + 1):
        for b in range(maxdeg + 1 - a):
            for c in range(maxdeg + 1 - a - b):
                val = np.sum(w * l1 ** a * l2 ** b * l3 ** c)
                assert val == pytest.approx(_bary_integral(a, b, c, area), rel=tol, abs=tol)


@pytest.mark.parametrize("rule", ["dunavant", "radon"])
def test_triangle_rules_degree_is_sharp(rule):
    """The stated degree is the largest: some monomial one degree higher is
    integrated with an error well above rounding."""
    A, B, C = np.array([0.0, 0, 0]), np.array([1.0, 0, 0]), np.array([0.0, 1, 0])
    pts, w = (dunavant4 if rule == "dunavant" else radon5)(A, B, C)
    d = 5 if rule == "dunavant" else 6
    T = np.stack([B - A, C - A], 1)
    lam = np.linalg.lstsq(T, (pts - A).T, rcond=None)[0].T
    l2, l3 = lam[:, 0], lam[:, 1]
    l1 = 1 - l2 - l3
    errs = [abs(np.sum(w * l1 ** a * l2 ** b * l3 ** (d - a - b)) - _bary_integral(a, b, d - a - b, 0.5))
            / _bary_integral(a, b, d - a - b, 0.5) for a in range(d + 1) for b in range(d + 1 - a)]
    assert max(errs) > 1e-6


def test_tet_rule_second_moments():
    """int_T x x^T = |T|/20 (sum_k p_k p_k^T + (sum p_k)(sum p_k)^T)."""
    rng = np.random.default_rng(1)
    P = rng.uniform(-1, 1, (4, 3))
    pts, w = tet_rule(*P, n=5)
    vol = np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]], 1)) / 6
    assert w.sum() == pytest.approx(vol, rel=1e-14)
    S = P.sum(0)
    ref = vol / 20 * (P.T @ P + np.outer(S, S))
    got = (w[:, None] * pts).T @ pts
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-15)


def test_unit_cube_cell():
    m = hex_mesh(1)
    c = cell_geometry(m, 0)
    assert c.volume == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(c.centroid, [0.5, 0.5, 0.5], atol=1e-14)
    assert c.diameter == pytest.approx(np.sqrt(3))
    # int (x - 1/2)^2 over the cube = 1/12
    Y = c.qp - 0.5
    assert np.sum(c.qw * Y[:, 0] ** 2) == pytest.approx(1 / 12, rel=1e-13)
    assert np.sum(c.qw * Y[:, 0] ** 2 * Y[:, 1] ** 2) == pytest.approx(1 / 144, rel=1e-13)
    # outward orientation: +x face of cell 0 points out, -x face in
    sig = {F.gid: F.sigma for F in c.faces}
    fs = m.cell_faces(0)
    assert sig[int(fs[0])] == -1 and sig[int(fs[1])] == 1


def test_affine_cell_moments():
    """An affine image of the unit cube: volume |det A|, centroid A c + b,
    second moments A (I/12) A^T |det A|."""
    A = np.array([[1.0, 0.3, 0.1], [0.0, 0.8, -0.2], [0.1, 0.0, 1.2]])
    b = np.array([0.2, -0.1, 0.4])
    m = affine(hex_mesh(1), A, b)
    c = cell_geometry(m, 0)
    det = np.linalg.det(A)
    assert c.volume == pytest.approx(det, rel=1e-14)
    np.testing.assert_allclose(c.centroid, A @ [0.5, 0.5, 0.5] + b, atol=1e-14)
    Y = c.qp - c.centroid
    np.testing.assert_allclose((c.qw[:, None] * Y).T @ Y, A @ A.T * det / 12, rtol=1e-12, atol=1e-15)


def test_face_geometry_square_and_triangle():
    m = hex_mesh(2)
    F = face_geometry(m, 0)
    assert F.area == pytest.approx(0.25)
    np.testing.assert_allclose(F.normal, [1, 0, 0])
    np.testing.assert_allclose(F.centroid, [0, 0.25, 0.25])
    assert F.diameter == pytest.approx(np.sqrt(2) / 2)
    assert abs(F.t1 @ F.normal) < 1e-15 and abs(F.t2 @ F.t1) < 1e-15
    t = tet_mesh(1)
    for f in range(t.n_faces):
        G = face_geometry(t, f)
        V = t.xyz[t.face_vertices(f)]
        assert G.area == pytest.approx(0.5 * np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[0])))
        np.testing.assert_allclose(G.centroid, V.mean(0), atol=1e-15)


def test_tet_mesh_volumes_sum_to_one():
    t = tet_mesh(2)
    vols = [cell_geometry(t, c).volume for c in range(t.n_cells)]
    assert sum(vols) == pytest.approx(1.0, rel=1e-13)
    np.testing.assert_allclose(vols, 1 / 48, rtol=1e-13)


def test_small_face_far_from_origin():
    """A triangle of side 1e-5 around (0.5, 0.7, 0.3), in a plane with a
    known unit normal: normal, area and centroid to rounding of the offsets
    (the area vector does not depend on the origin; computed about the
    vertex mean it keeps its digits)."""
    from synth.meshes import from_cell_loops
    nrm = np.array([1.0, 2.0, 2.0]) / 3.0
    t1 = np.array([2.0, -1.0, 0.0]) / np.sqrt(5.0)
    t2 = np.cross(nrm, t1)
    c0 = np.array([0.5, 0.7, 0.3])
    h = 1e-5
    tri = [c0 + h * t1, c0 + h * (-0.5 * t1 + 0.8 * t2), c0 + h * (-0.5 * t1 - 0.8 * t2)]
    apex = c0 - 0.1 * nrm
    xyz = np.array(tri + [apex])
    m = from_cell_loops(xyz, [[[0, 1, 2], [0, 1, 3], [1, 2, 3], [2, 0, 3]]])
    f = [i for i in range(m.n_faces) if sorted(m.face_vertices(i).tolist()) == [0, 1, 2]][0]
    F = face_geometry(m, f)
    np.testing.assert_allclose(F.normal, nrm, atol=1e-10)
    area = 0.5 * np.linalg.norm(np.cross(xyz[1] - xyz[0], xyz[2] - xyz[0]))
    assert F.area == pytest.approx(area, rel=1e-10)
    np.testing.assert_allclose(F.centroid, xyz[:3].mean(axis=0), atol=1e-15)
