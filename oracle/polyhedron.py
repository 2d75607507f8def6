"""Face and cell geometry of a polyhedral mesh (oracle).

Conventions (the paper leaves the face frame of Sec. 2, scaled face
monomials, unspecified; these are the project's readings):

* face global normal n_f: unit Newell normal of the stored vertex loop;
* face frame: t1 = (v1 - v0)/|v1 - v0| from the first two stored vertices,
  t2 = n_f x t1; both cells sharing a face use the same frame;
* |f|, x_f: area and area barycentre; h_f: largest vertex-vertex distance;
* |P|, x_P: volume and volume barycentre (Sec. 2, definition of m_alpha);
  h_P: largest vertex-vertex distance of the cell;
* sigma_{P,f} = +1 when n_f points out of P, else -1 (cells are convex, so
  the sign of (x_f - x_P) . n_f decides it).

Integration: faces are fanned into triangles (x_f, v_i, v_{i+1}); cells are
split into tetrahedra (x_ref, x_f, v_i, v_{i+1}) around the vertex mean
x_ref; both use the collapsed Gauss rules of quadrature.py.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .quadrature import cross3, triangle_rule, tet_rule


@dataclass
class Face:
    gid: int
    verts: np.ndarray      # (m, 3)
    normal: np.ndarray     # unit global normal
    area: float
    centroid: np.ndarray
    diameter: float
    t1: np.ndarray
    t2: np.ndarray
    sigma: int = 0         # orientation relative to the cell being processed
    bc: int = 0
    qp: np.ndarray = field(default=None, repr=False)   # exact-integration points
    qw: np.ndarray = field(default=None, repr=False)


@dataclass
class Cell:
    cid: int
    faces: list
    volume: float
    centroid: np.ndarray
    diameter: float
    qp: np.ndarray = field(default=None, repr=False)
    qw: np.ndarray = field(default=None, repr=False)


def face_geometry(mesh, f: int, nq: int = 5) -> Face:
    vid = mesh.face_vertices(f)
    V = mesh.xyz[vid]
    m = V.shape[0]
    # Newell: area vector = 1/2 sum v_i x v_{i+1}, the same for any origin
    # of the v_i (the loop is closed); taken about the vertex mean so that a
    # small face far from the origin loses no digits to cancellation
    xbar = V.mean(axis=0)
    W = V - xbar
    av = 0.5 * np.sum(np.cross(W, np.roll(W, -1, axis=0)), axis=0)
    a = np.linalg.norm(av)
    if not a > 0:
        raise ValueError(f"degenerate face {f}")
    n = av / a
    # area barycentre from the fan around the vertex mean
    num = np.zeros(3)
    den = 0.0
    for i in range(m):
        A, B = V[i], V[(i + 1) % m]
        sa = 0.5 * np.dot(cross3(A - xbar, B - xbar), n)
        num += sa * (xbar + A + B) / 3.0
        den += sa
    xf = num / den
    diam = max(np.linalg.norm(V[i] - V[j]) for i in range(m) for j in range(i + 1, m))
    t1 = (V[1] - V[0]) / np.linalg.norm(V[1] - V[0])
    t2 = cross3(n, t1)
    # exact-integration points: fan (x_f, v_i, v_{i+1})
    pts, wts = [], []
    for i in range(m):
        A, B = V[i], V[(i + 1) % m]
        p, w = triangle_rule(xf, A, B, nq)
        s = np.sign(np.dot(cross3(A - xf, B - xf), n))
        pts.append(p)
        wts.append(w * s)
    return Face(gid=f, verts=V, normal=n, area=den, centroid=xf, diameter=diam,
                t1=t1, t2=t2, bc=int(mesh.face_bc[f]),
                qp=np.concatenate(pts), qw=np.concatenate(wts))


def cell_geometry(mesh, c: int, faces_cache=None, nq: int = 5) -> Cell:
    fids = mesh.cell_faces(c)
    faces = []
    for f in fids:
        F = faces_cache[f] if faces_cache is not None else face_geometry(mesh, f, nq)
        faces.append(Face(**{k: getattr(F, k) for k in F.__dataclass_fields__}))
    allv = np.concatenate([F.verts for F in faces])
    uniq = np.unique(np.round(allv, 15), axis=0)
    xref = uniq.mean(axis=0)
    # orientation relative to this cell: outward iff normal points away from xref
    for F in faces:
        F.sigma = 1 if np.dot(F.centroid - xref, F.normal) > 0 else -1
    pts, wts = [], []
    for F in faces:
        m = F.verts.shape[0]
        for i in range(m):
            A, B = F.verts[i], F.verts[(i + 1) % m]
            p, w = tet_rule(xref, F.centroid, A, B, nq)
            # signed volume of (xref, x_f, A, B) is positive when the loop is
            # outward; flip for inward-oriented loops.
            pts.append(p)
            wts.append(w * F.sigma)
    qp = np.concatenate(pts)
    qw = np.concatenate(wts)
    vol = qw.sum()
    xc = (qw[:, None] * qp).sum(axis=0) / vol
    # re-check the orientation against the true barycentre
    for F in faces:
        s = 1 if np.dot(F.centroid - xc, F.normal) > 0 else -1
        if s != F.sigma:
            raise ValueError(f"cell {c}: face {F.gid} orientation ambiguous (non-convex cell?)")
    diam = 0.0
    for i in range(uniq.shape[0]):
        d = np.linalg.norm(uniq[i + 1:] - uniq[i], axis=1)
        if d.size:
            diam = max(diam, d.max())
    return Cell(cid=c, faces=faces, volume=vol, centroid=xc, diameter=diam, qp=qp, qw=qw)


def all_faces(mesh, nq: int = 5):
    return [face_geometry(mesh, f, nq) for f in range(mesh.n_faces)]
