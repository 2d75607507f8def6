"""Global assembly of the discrete problem eq. mod_prob_eqDisc (oracle).

Global numbering (the library's output layout, fixed by the C header):
  face DOF (f, beta)        -> nfd * f + beta
  interior DOF l of cell c  -> nfd * n_faces + nid * c + l
  pressure moment alpha     -> nq * c + alpha

The discrete problem  a_h(u, v) - b_h(v, p) = -<g_D, v.n>,  b_h(u, q) = (f, q)
is written with p~ = -p as the symmetric indefinite system
    [M  B^T] [u ]   [g]
    [B  0  ] [p~] = [F].
Face flags: 1 = Dirichlet pressure (natural, enters g); 2 (prescribed
flux) is not part of this oracle yet.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .element import ElementSpec, local_system
from .polyhedron import all_faces, cell_geometry


@dataclass
class System:
    spec: ElementSpec
    M: sp.csr_matrix
    B: sp.csr_matrix
    g: np.ndarray
    F: np.ndarray
    n_u: int
    n_p: int
    cells: list = field(repr=False, default=None)
    local: list = field(repr=False, default=None)
    dofmap: list = field(repr=False, default=None)

    @property
    def n(self) -> int:
        return self.n_u + self.n_p

    def saddle(self) -> sp.csr_matrix:
        return sp.bmat([[self.M, self.B.T], [self.B, None]], format="csr")

    def rhs(self) -> np.ndarray:
        return np.concatenate([self.g, self.F])


def cell_dofmap(mesh, c: int, spec: ElementSpec):
    nfd, nid = spec.nfd, spec.nid
    fs = mesh.cell_faces(c)
    idx = [nfd * int(f) + b for f in fs for b in range(nfd)]
    idx += [nfd * mesh.n_faces + nid * c + l for l in range(nid)]
    return np.array(idx, dtype=np.int64)


def assemble(mesh, spec: ElementSpec, nu_cell, f=None, gD=None, keep_local=False, nq=5) -> System:
    """Assemble M, B, g, F.  nu_cell = 1/K per cell (eq. bilin_form, nu = K^-1)."""
    if np.any(mesh.face_bc == 2):
        raise NotImplementedError("prescribed-flux faces")
    nu_cell = np.asarray(nu_cell, dtype=np.float64)
    faces = all_faces(mesh, nq)
    n_u = spec.nfd * mesh.n_faces + spec.nid * mesh.n_cells
    n_p = spec.nq * mesh.n_cells
    rows, cols, vals = [], [], []
    brows, bcols, bvals = [], [], []
    g = np.zeros(n_u)
    F = np.zeros(n_p)
    cells, locs, maps = [], [], []
    for c in range(mesh.n_cells):
        cell = cell_geometry(mesh, c, faces, nq)
        loc = local_system(cell, spec, float(nu_cell[c]), f=f, gD=gD)
        dm = cell_dofmap(mesh, c, spec)
        pm = spec.nq * c + np.arange(spec.nq)
        rows.append(np.repeat(dm, dm.size))
        cols.append(np.tile(dm, dm.size))
        vals.append(loc["M"].ravel())
        brows.append(np.repeat(pm, dm.size))
        bcols.append(np.tile(dm, pm.size))
        bvals.append(loc["B"].ravel())
        np.add.at(g, dm, loc["g"])
        F[pm] += loc["F"]
        if keep_local:
            cells.append(cell)
            locs.append(loc)
            maps.append(dm)
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n_u, n_u))
    B = sp.csr_matrix((np.concatenate(bvals), (np.concatenate(brows), np.concatenate(bcols))), shape=(n_p, n_u))
    M.sum_duplicates()
    B.sum_duplicates()
    return System(spec=spec, M=M, B=B, g=g, F=F, n_u=n_u, n_p=n_p,
                  cells=cells if keep_local else None,
                  local=locs if keep_local else None,
                  dofmap=maps if keep_local else None)


def mesh_cells(mesh, nq=5):
    faces = all_faces(mesh, nq)
    return [cell_geometry(mesh, c, faces, nq) for c in range(mesh.n_cells)]
