"""Global assembly of the discrete problem eq. mod_prob_eqDisc (oracle).

Global numbering (the library's output layout, fixed by the C header):
  face DOF (f, beta)        -> nfd * f + beta
  interior DOF l of cell c  -> nfd * n_faces + nid * c + l
  pressure moment alpha     -> nq * c + alpha

The discrete problem  a_h(u, v) - b_h(v, p) = -<g_D, v.n>,  b_h(u, q) = (f, q)
is written with p~ = -p as the symmetric indefinite system
    [M  B^T] [u ]   [g]
    [B  0  ] [p~] = [F].
Face flags: 1 = Dirichlet pressure (natural, enters g); 2 = prescribed normal
flux u.n = u_N (Sec. 3, the space V): the face DOFs of such a face are fixed
to the moments (1/|f|) int_f (u.n_f) m_beta of the given flux, the
corresponding rows and columns are eliminated (identity rows, their
coupling moved to the right-hand side).  With no Dirichlet face the pressure
lives in Q = {int q = 0} (Sec. 3): the mean-zero constraint enters through
one Lagrange multiplier, the "+1" of the paper's DOF counts,
    [M  B^T 0] [u ]   [g]
    [B  0   c] [p~] = [F],   c = (int_P psi_q)_(P,q),
    [0  c^T 0] [l ]   [0]
with psi_q the pressure basis dual to the moment DOFs (1/|P|) int_P p m_q
(eq. presMom): int_P psi_q = |P| for the constant moment, 0 for the others
(m_q has zero mean about the barycentre).  The constants have the moments
(1, 0, ..., 0) in every cell: that vector spans the kernel of B^T.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .element import ElementSpec, boundary_rule, local_system
from .polyhedron import all_faces, cell_geometry, face_geometry


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
    vol: np.ndarray = field(repr=False, default=None)          # cell volumes
    diam: np.ndarray = field(repr=False, default=None)         # cell diameters h_P
    fixed: np.ndarray = field(repr=False, default=None)        # prescribed flux DOFs
    fixed_val: np.ndarray = field(repr=False, default=None)
    multiplier: bool = False                                    # mean-zero pressure

    @property
    def n(self) -> int:
        return self.n_u + self.n_p

    def _full(self) -> sp.csr_matrix:
        return sp.bmat([[self.M, self.B.T], [self.B, None]], format="csr")

    def saddle(self) -> sp.csr_matrix:
        """[M B^T; B 0] with the prescribed flux DOFs eliminated (identity rows
        and zero columns)."""
        A = self._full()
        if self.fixed is None or self.fixed.size == 0:
            return A
        keep = np.ones(self.n)
        keep[self.fixed] = 0.0
        K = sp.diags(keep)
        return (K @ A @ K + sp.diags(1.0 - keep)).tocsr()

    def rhs(self) -> np.ndarray:
        b = np.concatenate([self.g, self.F])
        if self.fixed is None or self.fixed.size == 0:
            return b
        x0 = np.zeros(self.n)
        x0[self.fixed] = self.fixed_val
        b = b - self._full() @ x0
        b[self.fixed] = self.fixed_val
        return b

    @property
    def cvec(self) -> np.ndarray:
        """c_(P,q) = int_P psi_q: |P| on each cell's constant moment, 0 else."""
        nq = self.n_p // self.vol.size
        c = np.zeros(self.n_p)
        c[::nq] = self.vol
        return c

    @property
    def null_vec(self) -> np.ndarray:
        """The pressure moments of the constant 1 (kernel of B^T with the
        flux prescribed on the whole boundary)."""
        nq = self.n_p // self.vol.size
        e = np.zeros(self.n_p)
        e[::nq] = 1.0
        return e

    def augmented(self):
        """The system with the mean-zero multiplier row and column."""
        e = np.concatenate([np.zeros(self.n_u), self.cvec])[:, None]
        A = sp.bmat([[self.saddle(), sp.csr_matrix(e)], [sp.csr_matrix(e.T), None]], format="csr")
        return A, np.concatenate([self.rhs(), [0.0]])


def cell_dofmap(mesh, c: int, spec: ElementSpec):
    nfd, nid = spec.nfd, spec.nid
    fs = mesh.cell_faces(c)
    idx = [nfd * int(f) + b for f in fs for b in range(nfd)]
    idx += [nfd * mesh.n_faces + nid * c + l for l in range(nid)]
    return np.array(idx, dtype=np.int64)


def _cell_items(mesh, spec, nu, c, faces, f, gD, nq, bface_rule):
    """Geometry, local system and DOF map of cell c."""
    cell = cell_geometry(mesh, c, faces, nq)
    loc = local_system(cell, spec, float(nu), f=f, gD=gD, bface_rule=bface_rule)
    return cell, loc, cell_dofmap(mesh, c, spec)


def _cell_chunk(mesh, spec, nu_chunk, c0, c1, f, gD, nq, bface_rule):
    """_cell_items for the cells c0 .. c1 - 1 (in a worker process): the
    geometry of the faces these cells use is computed here, face by face as
    in all_faces, so every value is the one the sequential loop computes."""
    faces = {}
    for c in range(c0, c1):
        for fid in mesh.cell_faces(c):
            if int(fid) not in faces:
                faces[int(fid)] = face_geometry(mesh, int(fid), nq)
    return [_cell_items(mesh, spec, nu_chunk[c - c0], c, faces, f, gD, nq, bface_rule) for c in range(c0, c1)]


def _parallel_items(mesh, spec, nu_cell, f, gD, nq, bface_rule, processes):
    """Per-cell items in cell order from a pool of spawned processes (spawned,
    not forked, so a process that already uses a GPU can start it)."""
    import multiprocessing as mp
    from concurrent.futures import ProcessPoolExecutor
    nc = mesh.n_cells
    nchunk = min(nc, 8 * processes)
    bounds = [nc * i // nchunk for i in range(nchunk + 1)]
    with ProcessPoolExecutor(max_workers=processes, mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_cell_chunk, mesh, spec, nu_cell[a:b], a, b, f, gD, nq, bface_rule)
                for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        for fu in futs:
            yield from fu.result()


def assemble(mesh, spec: ElementSpec, nu_cell, f=None, gD=None, keep_local=False, nq=5, flux=None,
             bface_rule=None, processes: int = 1) -> System:
    """Assemble M, B, g, F.  nu_cell = 1/K per cell (eq. bilin_form, nu = K^-1).
    flux: the vector field u (callable (N,3) -> (N,3)) whose normal component
    is prescribed on faces with flag 2.  bface_rule: the fan rule of the
    boundary data (the Dirichlet term and the prescribed flux moments),
    'dunavant4' or 'radon5'; by default the library's, boundary_rule(spec).
    processes > 1 computes the per-cell local systems in that many spawned
    worker processes (f, gD must then be picklable, e.g. module-level
    functions); the global sums run in cell order either way, so the result
    is the same bit for bit."""
    if bface_rule is None:
        bface_rule = boundary_rule(spec)
    nu_cell = np.asarray(nu_cell, dtype=np.float64)
    n_u = spec.nfd * mesh.n_faces + spec.nid * mesh.n_cells
    n_p = spec.nq * mesh.n_cells
    rows, cols, vals = [], [], []
    brows, bcols, bvals = [], [], []
    g = np.zeros(n_u)
    F = np.zeros(n_p)
    cells, locs, maps = [], [], []
    vol = np.zeros(mesh.n_cells)
    diam = np.zeros(mesh.n_cells)
    if processes > 1 and mesh.n_cells > 1:
        items = _parallel_items(mesh, spec, nu_cell, f, gD, nq, bface_rule, processes)
        fl = np.nonzero(mesh.face_bc == 2)[0]
        faces = {int(fid): face_geometry(mesh, int(fid), nq) for fid in fl}
    else:
        faces = all_faces(mesh, nq)
        items = (_cell_items(mesh, spec, nu_cell[c], c, faces, f, gD, nq, bface_rule) for c in range(mesh.n_cells))
    for c, (cell, loc, dm) in enumerate(items):
        vol[c] = cell.volume
        diam[c] = cell.diameter
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
    fixed, fixed_val = prescribed_flux_dofs(mesh, spec, faces, flux, bface_rule)
    return System(spec=spec, M=M, B=B, g=g, F=F, n_u=n_u, n_p=n_p,
                  cells=cells if keep_local else None,
                  local=locs if keep_local else None,
                  dofmap=maps if keep_local else None,
                  vol=vol, diam=diam, fixed=fixed, fixed_val=fixed_val,
                  multiplier=bool(np.any(mesh.face_bc == 2)) and not bool(np.any(mesh.face_bc == 1)))


def prescribed_flux_dofs(mesh, spec: ElementSpec, faces, flux, rule=None):
    """Indices and values of the face DOFs fixed by the flux datum: on a face
    with flag 2, DOF (f, beta) = (1/|f|) int_f (u . n_f) m_beta^f with n_f
    the face's global normal and the boundary-data rule on the fan
    triangles (boundary_rule(spec) unless given)."""
    from .element import load_face_points
    from .monomials import eval_mono2, mono2
    fl = np.nonzero(mesh.face_bc == 2)[0]
    if fl.size == 0:
        return np.zeros(0, dtype=np.int64), np.zeros(0)
    if flux is None:
        raise ValueError("faces with flag 2 need the flux datum")
    betas = mono2(spec.kf)
    idx, val = [], []
    for f in fl:
        F = faces[f]
        pts, wts = load_face_points(F, rule or boundary_rule(spec))
        un = flux(pts) @ F.normal
        Mf = eval_mono2(betas, pts, F)
        mom = (wts * un) @ Mf / F.area
        for b in range(spec.nfd):
            idx.append(spec.nfd * int(f) + b)
            val.append(mom[b])
    return np.array(idx, dtype=np.int64), np.array(val)


def mesh_cells(mesh, nq=5):
    faces = all_faces(mesh, nq)
    return [cell_geometry(mesh, c, faces, nq) for c in range(mesh.n_cells)]
