"""Quadrature on triangles and tetrahedra (oracle).

Integration rules used to evaluate the exact polynomial integrals of the
method: collapsed (Duffy) tensor products of Gauss-Legendre points.  With n
points per direction the triangle rule integrates polynomials of total
degree <= 2n - 2 exactly and the tetrahedron rule degree <= 2n - 3.

The *load* rules (how f and g_D enter the right-hand side; the paper leaves
quadrature of data open, Sec. 4.3 remark on b_h and f_h) are fixed
conventions of this project, implemented here from their published
definitions and independently in the CUDA library:

* cell load rule for a P0 pressure: one point at the cell barycentre with
  weight |P| (the midpoint rule, exact for linear f);
* boundary-face rule: the face is fanned into triangles (x_f, v_i, v_{i+1})
  and each triangle gets, for E0 and the paper's k = 1, the 6-point
  degree-4 rule of D.A. Dunavant, "High degree efficient symmetrical
  Gaussian quadrature rules for the triangle", IJNME 21 (1985), Table for
  p = 4, and for k = 2 Radon's 7-point degree-5 rule, which makes the
  boundary data terms of the k = 2 element exact for cubic g_D (the
  library uses the same pair).
"""

from __future__ import annotations

from functools import lru_cache

import numpy as np
from numpy.polynomial.legendre import leggauss


def cross3(a, b):
    """Cross product of two 3-vectors (the componentwise products and
    differences of numpy.cross, without its general-shape overhead)."""
    return np.array([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


@lru_cache(maxsize=None)
def gauss01(n: int):
    """n-point Gauss-Legendre rule mapped to [0, 1] (memoised; read-only)."""
    x, w = leggauss(n)
    x, w = 0.5 * (x + 1.0), 0.5 * w
    x.flags.writeable = False
    w.flags.writeable = False
    return x, w


@lru_cache(maxsize=None)
def _ref_triangle(n: int):
    """Collapsed Gauss points (xi, eta) and weights on the unit right
    triangle {xi, eta >= 0, xi + eta <= 1}, weights summing to 1/2."""
    s, ws = gauss01(n)
    S, T = np.meshgrid(s, s, indexing="ij")
    WS, WT = np.meshgrid(ws, ws, indexing="ij")
    xi = S.ravel()
    eta = (T * (1.0 - S)).ravel()
    w = (WS * WT * (1.0 - S)).ravel()
    for a in (xi, eta, w):
        a.flags.writeable = False
    return xi, eta, w


@lru_cache(maxsize=None)
def _ref_tet(n: int):
    """Collapsed Gauss points (xi, eta, zeta) as an (N, 3) array and weights
    on the unit tetrahedron, weights summing to 1/6."""
    s, ws = gauss01(n)
    S, T, R = np.meshgrid(s, s, s, indexing="ij")
    WS, WT, WR = np.meshgrid(ws, ws, ws, indexing="ij")
    xi = S.ravel()
    eta = (T * (1.0 - S)).ravel()
    zeta = (R * (1.0 - S) * (1.0 - T)).ravel()
    w = (WS * WT * WR * (1.0 - S) ** 2 * (1.0 - T)).ravel()
    X = np.stack([xi, eta, zeta], 1)
    X.flags.writeable = False
    w.flags.writeable = False
    return X, w


def triangle_rule(A, B, C, n: int = 5):
    """Points (N,3) and weights (N,) on triangle ABC, |weights| summing to the area."""
    xi, eta, w = _ref_triangle(n)
    A = np.asarray(A, float)
    B = np.asarray(B, float)
    C = np.asarray(C, float)
    area2 = np.linalg.norm(cross3(B - A, C - A))
    pts = A[None, :] + xi[:, None] * (B - A)[None, :] + eta[:, None] * (C - A)[None, :]
    return pts, w * area2


def tet_rule(A, B, C, D, n: int = 5):
    """Points and *signed* weights on tetrahedron ABCD (sign of det[B-A, C-A, D-A])."""
    X, w = _ref_tet(n)
    A = np.asarray(A, float)
    J = np.stack([np.asarray(B, float) - A, np.asarray(C, float) - A, np.asarray(D, float) - A], 1)
    det = np.linalg.det(J)
    pts = A[None, :] + X @ J.T
    return pts, w * det


# Dunavant (1985) degree-4 rule, 6 points, barycentric (a, a, 1-2a) orbits;
# weights are fractions of the triangle area.
_DUN4_A = (0.445948490915965, 0.091576213509771)
_DUN4_W = (0.223381589678011, 0.109951743655322)


def dunavant4(A, B, C):
    """Dunavant degree-4 6-point rule on triangle ABC (points, area-weights)."""
    A = np.asarray(A, float)
    B = np.asarray(B, float)
    C = np.asarray(C, float)
    area = 0.5 * np.linalg.norm(cross3(B - A, C - A))
    bary = []
    wts = []
    for a, w in zip(_DUN4_A, _DUN4_W):
        b = 1.0 - 2.0 * a
        for l in ((a, a, b), (a, b, a), (b, a, a)):
            bary.append(l)
            wts.append(w)
    bary = np.array(bary)
    pts = bary[:, 0:1] * A + bary[:, 1:2] * B + bary[:, 2:3] * C
    return pts, np.array(wts) * area


def radon5(A, B, C):
    """Radon's degree-5 7-point rule on triangle ABC (J. Radon, "Zur
    mechanischen Kubatur", Monatsh. Math. 52 (1948)): the centroid with
    weight 9/40 and the orbits (a, a, 1 - 2a), a = (6 -+ sqrt 15)/21, with
    weights (155 -+ sqrt 15)/1200, as fractions of the area."""
    A = np.asarray(A, float)
    B = np.asarray(B, float)
    C = np.asarray(C, float)
    area = 0.5 * np.linalg.norm(cross3(B - A, C - A))
    r15 = np.sqrt(15.0)
    bary = [(1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0)]
    wts = [9.0 / 40.0]
    for a, w in (((6.0 - r15) / 21.0, (155.0 - r15) / 1200.0), ((6.0 + r15) / 21.0, (155.0 + r15) / 1200.0)):
        b = 1.0 - 2.0 * a
        for l in ((a, a, b), (a, b, a), (b, a, a)):
            bary.append(l)
            wts.append(w)
    bary = np.array(bary)
    pts = bary[:, 0:1] * A + bary[:, 1:2] * B + bary[:, 2:3] * C
    return pts, np.array(wts) * area
