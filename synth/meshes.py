"""Polyhedral meshes of the unit cube, as plain topology + coordinates.

A mesh is face based, which is all the mixed virtual element space needs
(its degrees of freedom live on faces and in cells, none on vertices or
edges):

* ``xyz``            (n_vertices, 3) float64 vertex coordinates;
* ``face_vtx_ptr``   (n_faces + 1,) int64 and ``face_vtx`` int32: the vertex
  loop of each planar face.  The loop orientation fixes the face's global
  normal by the right-hand rule;
* ``cell_face_ptr``  (n_cells + 1,) int64 and ``cell_face`` int32: the faces of
  each cell;
* ``face_bc``        (n_faces,) int8: 0 interior, 1 Dirichlet pressure,
  2 prescribed normal flux.

The first two vertices of a face also fix its in-plane frame (the face's
local x axis points from the first to the second vertex).
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class Mesh:
    xyz: np.ndarray
    face_vtx_ptr: np.ndarray
    face_vtx: np.ndarray
    cell_face_ptr: np.ndarray
    cell_face: np.ndarray
    face_bc: np.ndarray
    name: str = ""

    @property
    def n_vertices(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_faces(self) -> int:
        return int(self.face_vtx_ptr.shape[0] - 1)

    @property
    def n_cells(self) -> int:
        return int(self.cell_face_ptr.shape[0] - 1)

    def face_vertices(self, f: int) -> np.ndarray:
        return self.face_vtx[self.face_vtx_ptr[f]:self.face_vtx_ptr[f + 1]]

    def cell_faces(self, c: int) -> np.ndarray:
        return self.cell_face[self.cell_face_ptr[c]:self.cell_face_ptr[c + 1]]

    def validate(self) -> None:
        assert self.xyz.dtype == np.float64 and self.xyz.ndim == 2 and self.xyz.shape[1] == 3
        assert self.face_vtx_ptr.dtype == np.int64 and self.cell_face_ptr.dtype == np.int64
        assert self.face_vtx.dtype == np.int32 and self.cell_face.dtype == np.int32
        assert self.face_bc.dtype == np.int8 and self.face_bc.shape == (self.n_faces,)
        assert self.face_vtx_ptr[0] == 0 and self.face_vtx_ptr[-1] == self.face_vtx.size
        assert self.cell_face_ptr[0] == 0 and self.cell_face_ptr[-1] == self.cell_face.size
        assert np.all(np.diff(self.face_vtx_ptr) >= 3)
        assert np.all(np.diff(self.cell_face_ptr) >= 4)
        # every face belongs to one (boundary) or two (interior) cells
        cnt = np.bincount(self.cell_face, minlength=self.n_faces)
        assert np.all((cnt == 1) | (cnt == 2)), "face shared by more than two cells"
        assert np.all((cnt == 1) == (self.face_bc != 0)), "boundary flags disagree with adjacency"


def hex_mesh(n: int, bc: int = 1) -> Mesh:
    """Structured n x n x n mesh of [0,1]^3 by cubes.

    Faces are numbered x-normal first (plane index i, then j, k), then
    y-normal, then z-normal; every face's global normal is the +axis.
    Cells are numbered (i*n + j)*n + k with i the x index; each cell lists
    its faces as -x, +x, -y, +y, -z, +z.  Boundary faces get flag ``bc``.
    """
    if n < 1:
        raise ValueError("n >= 1")
    m = n + 1
    g = np.linspace(0.0, 1.0, m)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1).astype(np.float64)

    def vid(i, j, k):
        return (i * m + j) * m + k

    I, J, K = np.meshgrid(np.arange(m), np.arange(n), np.arange(n), indexing="ij")
    I, J, K = I.ravel(), J.ravel(), K.ravel()
    # x-faces at plane i: loop (j,k) -> (j+1,k) -> (j+1,k+1) -> (j,k+1): normal +x
    fx = np.stack([vid(I, J, K), vid(I, J + 1, K), vid(I, J + 1, K + 1), vid(I, J, K + 1)], 1)
    bx = (I == 0) | (I == n)
    # y-faces at plane j (index order i, j, k with j the plane): normal +y
    Iy, Jy, Ky = np.meshgrid(np.arange(n), np.arange(m), np.arange(n), indexing="ij")
    Iy, Jy, Ky = Iy.ravel(), Jy.ravel(), Ky.ravel()
    fy = np.stack([vid(Iy, Jy, Ky), vid(Iy, Jy, Ky + 1), vid(Iy + 1, Jy, Ky + 1), vid(Iy + 1, Jy, Ky)], 1)
    by = (Jy == 0) | (Jy == n)
    # z-faces at plane k: normal +z
    Iz, Jz, Kz = np.meshgrid(np.arange(n), np.arange(n), np.arange(m), indexing="ij")
    Iz, Jz, Kz = Iz.ravel(), Jz.ravel(), Kz.ravel()
    fz = np.stack([vid(Iz, Jz, Kz), vid(Iz + 1, Jz, Kz), vid(Iz + 1, Jz + 1, Kz), vid(Iz, Jz + 1, Kz)], 1)
    bz = (Kz == 0) | (Kz == n)

    faces = np.concatenate([fx, fy, fz], 0).astype(np.int32)
    nfx = fx.shape[0]
    nfy = fy.shape[0]
    face_bc = np.where(np.concatenate([bx, by, bz]), bc, 0).astype(np.int8)

    ci, cj, ck = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()

    def xf(i, j, k):
        return (i * n + j) * n + k

    def yf(i, j, k):
        return nfx + (i * m + j) * n + k

    def zf(i, j, k):
        return nfx + nfy + (i * n + j) * m + k

    cf = np.stack([xf(ci, cj, ck), xf(ci + 1, cj, ck),
                   yf(ci, cj, ck), yf(ci, cj + 1, ck),
                   zf(ci, cj, ck), zf(ci, cj, ck + 1)], 1).astype(np.int32)

    mesh = Mesh(
        xyz=xyz,
        face_vtx_ptr=np.arange(0, 4 * faces.shape[0] + 1, 4, dtype=np.int64),
        face_vtx=faces.ravel().copy(),
        cell_face_ptr=np.arange(0, 6 * cf.shape[0] + 1, 6, dtype=np.int64),
        cell_face=cf.ravel().copy(),
        face_bc=face_bc,
        name=f"hex{n}",
    )
    return mesh


def cell_vertex_ids(mesh: Mesh, c: int) -> np.ndarray:
    """Distinct vertex ids of cell c (union over its faces)."""
    fs = mesh.cell_faces(c)
    return np.unique(np.concatenate([mesh.face_vertices(f) for f in fs]))


def from_cell_loops(xyz: np.ndarray, cells, boundary_bc: int = 1, name: str = "") -> Mesh:
    """Build a Mesh from cells given as lists of vertex loops (any orientation).

    Loops are matched across cells by their vertex set; the first cell that
    lists a face fixes its stored loop, oriented outward from that cell.
    Faces listed by one cell only get flag ``boundary_bc``.
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    key2face = {}
    loops = []
    count = []
    cell_face = []
    ptr = [0]
    for cl in cells:
        allv = np.unique(np.concatenate([np.asarray(l) for l in cl]))
        ctr = xyz[allv].mean(axis=0)
        for loop in cl:
            loop = [int(v) for v in loop]
            key = tuple(sorted(loop))
            if key not in key2face:
                P = xyz[loop]
                av = 0.5 * np.sum(np.cross(P, np.roll(P, -1, axis=0)), axis=0)
                if np.dot(P.mean(axis=0) - ctr, av) < 0:
                    loop = loop[::-1]
                key2face[key] = len(loops)
                loops.append(loop)
                count.append(0)
            fid = key2face[key]
            count[fid] += 1
            cell_face.append(fid)
        ptr.append(len(cell_face))
    fptr = np.zeros(len(loops) + 1, dtype=np.int64)
    fptr[1:] = np.cumsum([len(l) for l in loops])
    mesh = Mesh(xyz=xyz, face_vtx_ptr=fptr,
                face_vtx=np.concatenate([np.asarray(l) for l in loops]).astype(np.int32),
                cell_face_ptr=np.asarray(ptr, dtype=np.int64),
                cell_face=np.asarray(cell_face, dtype=np.int32),
                face_bc=np.where(np.asarray(count) == 1, boundary_bc, 0).astype(np.int8),
                name=name)
    mesh.validate()
    return mesh


def _grid_vertices(n: int):
    m = n + 1
    g = np.linspace(0.0, 1.0, m)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(i, j, k):
        return (i * m + j) * m + k
    return xyz, vid


def tet_mesh(n: int, bc: int = 1) -> Mesh:
    """Kuhn subdivision: every cube of an n^3 grid split into 6 tetrahedra
    around its main diagonal (conforming across cubes)."""
    xyz, vid = _grid_vertices(n)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    cells = []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                for pm in perms:
                    p = [0, 0, 0]
                    vs = [vid(i, j, k)]
                    for ax in pm:
                        p[ax] += 1
                        vs.append(vid(i + p[0], j + p[1], k + p[2]))
                    cells.append([[vs[a] for a in range(4) if a != skip] for skip in range(4)])
    return from_cell_loops(xyz, cells, bc, name=f"tet{n}")


def prism_mesh(n: int, bc: int = 1) -> Mesh:
    """Every cube of an n^3 grid split by its x = y diagonal plane into two
    triangular prisms (triangle and quadrilateral faces)."""
    xyz, vid = _grid_vertices(n)
    cells = []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                a0, b0, c0, d0 = vid(i, j, k), vid(i + 1, j, k), vid(i + 1, j + 1, k), vid(i, j + 1, k)
                a1, b1, c1, d1 = vid(i, j, k + 1), vid(i + 1, j, k + 1), vid(i + 1, j + 1, k + 1), vid(i, j + 1, k + 1)
                for (p, q, r), (p1, q1, r1) in (((a0, b0, c0), (a1, b1, c1)), ((a0, c0, d0), (a1, c1, d1))):
                    cells.append([[p, q, r], [p1, q1, r1], [p, q, q1, p1], [q, r, r1, q1], [r, p, p1, r1]])
    return from_cell_loops(xyz, cells, bc, name=f"prism{n}")


def octa_mesh(n: int, bc: int = 1) -> Mesh:
    """Every cube of an n^3 grid split into 9 convex cells: the octahedron
    whose vertices are the 6 face centres of the cube (8 triangular faces),
    and the 8 corner pieces {cube octant} minus that octahedron, each with 7
    faces (the quarter squares of the 3 cube faces at its corner, a triangle
    on each of the 3 mid-planes, a triangle on the octahedron).  Cells have
    seven or eight faces; 9 n^3 cells, 20 n^3 + 12 n^2 (n + 1) faces and the
    (2n+1)^3 points of the half-step grid as vertices."""
    m = 2 * n + 1
    g = np.linspace(0.0, 1.0, m)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def vid(p):
        return (p[0] * m + p[1]) * m + p[2]
    e = np.eye(3, dtype=np.int64)
    cells = []
    for i in range(n):
        for j in range(n):
            for k in range(n):
                C = np.array([2 * i + 1, 2 * j + 1, 2 * k + 1])
                cells.append([[vid(C + sx * e[0]), vid(C + sy * e[1]), vid(C + sz * e[2])]
                              for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)])
                for sx in (-1, 1):
                    for sy in (-1, 1):
                        for sz in (-1, 1):
                            Fx, Fy, Fz = C + sx * e[0], C + sy * e[1], C + sz * e[2]
                            Exy, Exz, Eyz = Fx + sy * e[1], Fx + sz * e[2], Fy + sz * e[2]
                            V = Exy + sz * e[2]
                            cells.append([[vid(Fx), vid(Exy), vid(V), vid(Exz)],
                                          [vid(Fy), vid(Exy), vid(V), vid(Eyz)],
                                          [vid(Fz), vid(Exz), vid(V), vid(Eyz)],
                                          [vid(Fy), vid(Fz), vid(Eyz)],
                                          [vid(Fx), vid(Fz), vid(Exz)],
                                          [vid(Fx), vid(Fy), vid(Exy)],
                                          [vid(Fx), vid(Fy), vid(Fz)]])
    return from_cell_loops(xyz, cells, bc, name=f"octa{n}")


def affine(mesh: Mesh, A, b=(0.0, 0.0, 0.0)) -> Mesh:
    """Image of a mesh under x -> A x + b (faces stay planar)."""
    A = np.asarray(A, dtype=np.float64)
    out = Mesh(xyz=mesh.xyz @ A.T + np.asarray(b, dtype=np.float64),
               face_vtx_ptr=mesh.face_vtx_ptr.copy(), face_vtx=mesh.face_vtx.copy(),
               cell_face_ptr=mesh.cell_face_ptr.copy(), cell_face=mesh.cell_face.copy(),
               face_bc=mesh.face_bc.copy(), name=mesh.name + "_affine")
    return out
