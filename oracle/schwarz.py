"""Edge-patch additive Schwarz smoothing for the regularised flux block
A_reg = A + B^T W^-1 B of Block-Reg (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

A_reg is a discrete grad-div operator: fields with small divergence have
small energy, and at the paper's k = 2 many of them live inside a few cells
(interior gradient and cross moments with P2 face moments).  Point smoothers
leave those errors in place and a scalar aggregation cannot represent them
on the coarse grid.  The remedy of D. N. Arnold, R. S. Falk, R. Winther,
"Multigrid in H(div) and H(curl)", Numer. Math. 85 (2000) is a Schwarz
smoother over patches that contain the supports of the local
divergence-free fields; in three dimensions those are the patches of the
cells around a mesh edge.  Here:

* edge patch of the edge (v, w): the flux DOFs of every face whose vertex
  loop has v and w as neighbours, and the interior DOFs of every cell that
  has one of those faces; DOF indices sorted increasingly;
* additive Schwarz operator M_S = sum_i R_i^T (R_i A R_i^T)^-1 R_i over the
  patches (R_i the restriction to patch i);
* smoother weight omega_S = 4 / (3 rho_S), rho_S = 1.1 x the largest Ritz
  value of M_S A after 10 Lanczos steps in the A-inner product (M_S A is
  self-adjoint there) from the SplitMix64 start vector of
  ``block_amg.start_vector``;
* V-cycle: the hierarchy of ``amg.setup`` (damped-Jacobi smoothing on the
  coarse levels), with the finest level smoothed by omega_S M_S before and
  after the coarse correction: x = omega_S M_S b;
  x += P V_1(P^T (b - A x)); x += omega_S M_S (b - A x).  The cycle is
  symmetric, and positive definite when omega_S rho(M_S A) < 2.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from . import amg
from .block_amg import start_vector


def edges_and_faces(mesh):
    """Map each edge (v, w), v < w, to the faces whose loops contain it."""
    out = {}
    for f in range(mesh.n_faces):
        v = mesh.face_vertices(f)
        for i in range(len(v)):
            a, b = int(v[i]), int(v[(i + 1) % len(v)])
            out.setdefault((min(a, b), max(a, b)), []).append(f)
    return out


def edge_patches(mesh, spec):
    """DOF index arrays of the edge patches, in edge order (sorted pairs)."""
    face_cells = [[] for _ in range(mesh.n_faces)]
    for c in range(mesh.n_cells):
        for f in mesh.cell_faces(c):
            face_cells[int(f)].append(c)
    base = spec.nfd * mesh.n_faces
    patches = []
    for _, fs in sorted(edges_and_faces(mesh).items()):
        cells = sorted({c for f in fs for c in face_cells[f]})
        dofs = [spec.nfd * f + b for f in fs for b in range(spec.nfd)]
        dofs += [base + spec.nid * c + l for c in cells for l in range(spec.nid)]
        patches.append(np.array(sorted(dofs), dtype=np.int64))
    return patches


def schwarz_operator(A: sp.csr_matrix, patches) -> sp.csr_matrix:
    """M_S = sum_i R_i^T (R_i A R_i^T)^-1 R_i."""
    A = A.tocsr()
    rows, cols, vals = [], [], []
    for G in patches:
        inv = np.linalg.inv(A[G][:, G].toarray())
        r, c = np.meshgrid(G, G, indexing="ij")
        rows.append(r.ravel())
        cols.append(c.ravel())
        vals.append(inv.ravel())
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=A.shape)
    M.sum_duplicates()
    return M


def lanczos_max_A(A: sp.csr_matrix, MS: sp.csr_matrix, steps: int = 10) -> float:
    """Largest Ritz value of M_S A after ``steps`` Lanczos steps in the
    A-inner product with full reorthogonalisation (a lower bound of
    lambda_max(M_S A))."""
    n = A.shape[0]
    V = np.zeros((n, steps + 1))
    v = start_vector(n)
    V[:, 0] = v / np.sqrt(v @ (A @ v))
    alpha, beta = [], []
    for k in range(steps):
        w = MS @ (A @ V[:, k])
        Aw = A @ w
        a = V[:, k] @ Aw
        AV = A @ V[:, :k + 1]
        w = w - V[:, :k + 1] @ (AV.T @ w)
        alpha.append(a)
        b = np.sqrt(max(w @ (A @ w), 0.0))
        if b <= 1e-12 * abs(a) or k == steps - 1:
            break
        beta.append(b)
        V[:, k + 1] = w / b
    m = len(alpha)
    T = np.diag(alpha) + np.diag(beta[:m - 1], 1) + np.diag(beta[:m - 1], -1)
    return float(np.linalg.eigvalsh(T).max())


@dataclass
class SchwarzCycle:
    H: amg.Hierarchy
    MS: sp.csr_matrix
    omega: float
    rho: float

    def __call__(self, b: np.ndarray) -> np.ndarray:
        lv = self.H.levels[0]
        if len(self.H.levels) == 1:
            return amg.coarse_solve(self.H, b)
        x = self.omega * (self.MS @ b)
        x = x + lv.P @ amg.vcycle(self.H, lv.P.T @ (b - lv.A @ x), 1)
        return x + self.omega * (self.MS @ (b - lv.A @ x))


def setup(A: sp.csr_matrix, patches, **amg_kw) -> SchwarzCycle:
    A = A.tocsr()
    H = amg.setup(A, smoother="jacobi", **amg_kw)
    MS = schwarz_operator(A, patches)
    rho = 1.1 * lanczos_max_A(A, MS)
    return SchwarzCycle(H=H, MS=MS, omega=4.0 / (3.0 * rho), rho=rho)
