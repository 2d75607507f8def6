"""Smoothed aggregation on point blocks, for a Schur block S with several
pressure DOFs per cell (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

For the paper's k = 2 element every cell carries the four P1 pressure
moments (eq. presMom), and S = B diag(M)^-1 B^T couples the moments of a cell
and of its face neighbours in 4 x 4 blocks.  The scalar aggregation of
``oracle/amg.py`` then splits the moments of one cell over different
aggregates, and its coarse space holds only piecewise-constant vectors of
moments, which are not smooth pressures.  This module keeps a cell's block
together and builds the coarse space from the pressures that S leaves
nearly unchanged -- the moments of 1, x, y and z -- following

* P. Vanek, J. Mandel, M. Brezina, "Algebraic multigrid by smoothed
  aggregation for second and fourth order elliptic problems", Computing 56
  (1996): tentative prolongator from a near-null space B, orthonormalised
  per aggregate (T R = B restricted to the aggregate), coarse near-null
  space R, prolongator smoothing P = (I - omega D^-1 A) T;
* the aggregation (strength, distance-2 MIS, the three passes) of
  ``oracle/amg.py``, applied to the graph of the blocks.

Exact rules:

* block norm N_IJ = Frobenius norm of the bs x bs block (I, J) of A;
  strong(I, J): J != I and N_IJ >= theta sqrt(N_II N_JJ);
* aggregates: ``amg.aggregate`` on that graph (isolated blocks stay out of
  the coarse space); an aggregate on which B has numerical rank below m (a
  Cholesky pivot of B_a^T B_a at most 1e-10 of its diagonal entry) is
  dissolved, its blocks left out of the coarse space, and the others are
  renumbered in order (``dissolve_rank_deficient``; the paper uses PETSc's
  GAMG and does not describe its coarse spaces, so this rule is ours);
* T: for aggregate a with member blocks I_1 < I_2 < ..., the rows of its
  DOFs (block by block, component by component) of B have the thin QR
  factorisation Q R with R upper triangular and R_jj > 0 (unique for full
  column rank); T holds Q in columns a m .. a m + m - 1, the coarse B holds R
  in rows a m .. a m + m - 1 (m = columns of B);
* D = block diagonal of A (bs x bs blocks), D = L L^T blockwise
  (Cholesky); C = L^-1 A L^-T is symmetric and similar to D^-1 A;
* rho = min(G, 1.1 theta): G = max_i sum_j |C_ij| (Gershgorin, an upper
  bound of the spectrum of D^-1 A), theta = the largest Ritz value of C
  after 10 Lanczos steps from a SplitMix64 start vector (a lower bound that
  approaches lambda_max quickly).  On the k = 2 Schur block, whose moment
  DOFs of one cell differ in scale by two orders of magnitude, the row sums
  of D^-1 A overshoot lambda_max about six times and those of C still 1.5
  (cubes) to 2.6 times (CVT), damping the smoother that much too strongly;
  PETSc's GAMG likewise scales a Krylov estimate by 1.1.
  omega = 4 / (3 rho); the damped block-Jacobi error factor 1 - omega lambda
  stays in (-1, 1) whenever rho > 2/3 lambda_max;
* P = T - omega D^-1 A T (prolongator smoothing with the full A);
* coarse matrix P^T A P, block size m, theta halved per level; stop rules
  and the coarsest solve as in ``amg.setup`` (counted in blocks);
* cycle: V(1,1) with damped block Jacobi, x = omega D^-1 b;
  x += P V(P^T (b - A x)); x += omega D^-1 (b - A x); symmetric, and
  positive definite when the smoother converges (rho > 2/3 lambda_max).
  Or (smoother='chebyshev') two Chebyshev steps of block Jacobi on
  [rho/10, rho] before and after the coarse correction.

The same construction serves the regularised flux block A_reg of Block-Reg:
at the paper's k = 1 directly, whose face moments (3 per face) and interior
moments (3 per cell) form 3 x 3 blocks, and at any k >= 1 on the face system
left after eliminating the interior DOFs cell by cell (``CondensedCycle``),
with the DOFs of the three constant vector fields as near-null space
(``flux_modes``) and Chebyshev smoothing.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from . import amg
from .solvers import Result


def block_norms(A: sp.csr_matrix, bs: int) -> sp.csr_matrix:
    """N_IJ = Frobenius norm of block (I, J)."""
    C = A.tocoo()
    nb = A.shape[0] // bs
    N = sp.csr_matrix((C.data ** 2, (C.row // bs, C.col // bs)), shape=(nb, nb))
    N.sum_duplicates()
    N.data = np.sqrt(N.data)
    return N


def block_strength(A: sp.csr_matrix, bs: int, theta: float):
    """Strong neighbour lists of the block graph (CSR pointer and indices)."""
    N = block_norms(A, bs)
    d = N.diagonal()
    ptr = [0]
    idx = []
    for i in range(N.shape[0]):
        for k in range(N.indptr[i], N.indptr[i + 1]):
            j = int(N.indices[k])
            if j != i and N.data[k] >= theta * np.sqrt(d[i] * d[j]):
                idx.append(j)
        ptr.append(len(idx))
    return np.array(ptr, dtype=np.int64), np.array(idx, dtype=np.int64)


def diag_blocks(A: sp.csr_matrix, bs: int):
    A = A.tocsr()
    return [A[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs].toarray() for i in range(A.shape[0] // bs)]


def block_diag_inv(A: sp.csr_matrix, bs: int) -> sp.csr_matrix:
    return sp.block_diag([sp.csr_matrix(np.linalg.inv(D)) for D in diag_blocks(A, bs)], format="csr")


def symmetric_form(A: sp.csr_matrix, bs: int) -> sp.csr_matrix:
    """L^-1 A L^-T with D = L L^T (Cholesky of every diagonal block): the
    symmetric matrix similar to D^-1 A = L^-T (L^-1 A L^-T) L^T."""
    Linv = sp.block_diag([sp.csr_matrix(np.linalg.inv(np.linalg.cholesky(D))) for D in diag_blocks(A, bs)],
                         format="csr")
    return (Linv @ A @ Linv.T).tocsr()


def start_vector(n: int) -> np.ndarray:
    """v_i = 2 u_i - 1, u_i = the top 53 bits of splitmix64(i) / 2^53."""
    return np.array([2.0 * (amg.splitmix64(i) >> 11) / 2.0 ** 53 - 1.0 for i in range(n)])


def lanczos_max(C: sp.csr_matrix, steps: int) -> float:
    """Largest Ritz value of C after ``steps`` Lanczos steps from
    start_vector (C. Lanczos, J. Res. NBS 45 (1950)), with full
    reorthogonalisation; a lower bound of lambda_max(C)."""
    n = C.shape[0]
    V = np.zeros((n, steps + 1))
    v = start_vector(n)
    V[:, 0] = v / np.linalg.norm(v)
    alpha, beta = [], []
    k = 0
    for k in range(steps):
        w = C @ V[:, k]
        a = V[:, k] @ w
        w = w - V[:, :k + 1] @ (V[:, :k + 1].T @ w)
        alpha.append(a)
        b = np.linalg.norm(w)
        if b <= 1e-12 * abs(a) or k == steps - 1:
            break
        beta.append(b)
        V[:, k + 1] = w / b
    Tk = np.diag(alpha) + np.diag(beta[:len(alpha) - 1], 1) + np.diag(beta[:len(alpha) - 1], -1)
    return float(np.linalg.eigvalsh(Tk).max())


def rho_estimate(A: sp.csr_matrix, bs: int, steps: int = 10, safety: float = 1.1) -> float:
    """Estimate of the spectral radius of D^-1 A: min(Gershgorin bound of the
    symmetric form, safety x its largest Ritz value after ``steps`` Lanczos
    steps).  The row sums bound the spectrum but overshoot it several times
    for moment DOFs of different scales; the Ritz value approaches it from
    below (PETSc's GAMG likewise scales a Krylov estimate by 1.1)."""
    C = symmetric_form(A, bs)
    gersh = float(np.asarray(abs(C).sum(axis=1)).max())
    if C.shape[0] <= steps:
        return min(gersh, safety * float(np.linalg.eigvalsh(C.toarray()).max()))
    return min(gersh, safety * lanczos_max(C, steps))


def qr_positive(X: np.ndarray):
    """Thin QR with a positive diagonal of R (unique for full column rank)."""
    Q, R = np.linalg.qr(X)
    s = np.sign(np.diag(R))
    if np.any(s == 0.0):
        raise np.linalg.LinAlgError("near-null space rank-deficient on an aggregate")
    return Q * s, s[:, None] * R


RANK_TOL = 1e-10


def dissolve_rank_deficient(agg: np.ndarray, nc: int, B: np.ndarray, bs: int, tol: float = RANK_TOL):
    """Aggregates on which the near-null space has numerical rank below its
    width m are dissolved: their blocks leave the coarse space (agg = -1,
    like blocks without strong neighbours) and the remaining aggregates are
    renumbered in their order.  Rank test: a pivot of the Cholesky
    factorisation of the Gram matrix G = B_a^T B_a, d_j = G_jj - sum_{k<j}
    R_kj^2, at most tol G_jj.  (A face aggregate of Block-Reg's condensed
    system with fewer than three independent face normals has rank < 3 on
    the constant fields; without this rule its QR gives a column of rounding
    noise.)"""
    m = B.shape[1]
    keep = np.zeros(nc, dtype=bool)
    for a in range(nc):
        members = np.nonzero(agg == a)[0]
        dofs = (members[:, None] * bs + np.arange(bs)[None, :]).ravel()
        G = B[dofs].T @ B[dofs]
        R = np.zeros((m, m))
        ok = True
        for j in range(m):
            d = G[j, j] - R[:j, j] @ R[:j, j]
            if not d > tol * G[j, j]:
                ok = False
                break
            R[j, j] = np.sqrt(d)
            for i in range(j + 1, m):
                R[j, i] = (G[j, i] - R[:j, j] @ R[:j, i]) / R[j, j]
        keep[a] = ok
    new_id = np.cumsum(keep) - 1
    out = np.where((agg >= 0) & keep[np.maximum(agg, 0)], new_id[np.maximum(agg, 0)], -1)
    return out.astype(agg.dtype), int(keep.sum())


def tentative(agg: np.ndarray, nc: int, B: np.ndarray, bs: int):
    """T (n x nc m) and the coarse near-null space (nc m x m)."""
    n, m = B.shape
    rows, cols, vals = [], [], []
    Bc = np.zeros((nc * m, m))
    for a in range(nc):
        members = np.nonzero(agg == a)[0]
        dofs = (members[:, None] * bs + np.arange(bs)[None, :]).ravel()
        Q, R = qr_positive(B[dofs])
        rows.append(np.repeat(dofs, m))
        cols.append(np.tile(a * m + np.arange(m), dofs.size))
        vals.append(Q.ravel())
        Bc[a * m:(a + 1) * m] = R
    T = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, nc * m))
    return T, Bc


@dataclass
class Level:
    A: sp.csr_matrix
    bs: int
    Dinv: sp.csr_matrix
    omega: float
    rho: float
    agg: np.ndarray = None
    P: sp.csr_matrix = None


@dataclass
class Hierarchy:
    levels: list = field(default_factory=list)
    coarse_inv: np.ndarray = None
    smoother: str = "jacobi"           # 'jacobi' (one damped step) or 'chebyshev'
    degree: int = 2                    # Chebyshev steps per smoothing

    @property
    def sizes(self):
        return [lv.A.shape[0] for lv in self.levels]


def setup(A: sp.csr_matrix, bs: int, B: np.ndarray, theta: float = 0.08, coarse_max: int = 64,
          max_levels: int = 12, dense_max: int = 1024, pin_last: bool = False,
          smoother: str = "jacobi", degree: int = 2) -> Hierarchy:
    """A: SPD with bs x bs point blocks, or SPSD with the constant pressure
    as null space (pin_last: flux data on the whole boundary; its first
    column of B must be that null vector); B: near-null space, one row per
    DOF of A.  smoother: damped block Jacobi, or 'chebyshev': ``degree``
    steps of Chebyshev acceleration of block Jacobi on [rho/10, rho] (Saad
    2003, Algorithm 12.1, as in ``amg.chebyshev`` with D the block
    diagonal); the hierarchy does not depend on it."""
    if smoother not in ("jacobi", "chebyshev"):
        raise ValueError(smoother)
    A = A.tocsr()
    B = np.asarray(B, dtype=np.float64)
    if A.shape[0] % bs or B.shape[0] != A.shape[0]:
        raise ValueError("A and B must consist of whole blocks")
    H = Hierarchy(smoother=smoother, degree=degree)
    th = theta
    while True:
        Dinv = block_diag_inv(A, bs)
        rho = rho_estimate(A, bs)
        lv = Level(A=A, bs=bs, Dinv=Dinv, omega=4.0 / (3.0 * rho), rho=rho)
        H.levels.append(lv)
        nb = A.shape[0] // bs
        if nb <= coarse_max or len(H.levels) == max_levels:
            break
        ptr, idx = block_strength(A, bs, th)
        agg, nc = amg.aggregate(nb, ptr, idx)
        if nc == 0 or 5 * nc > 4 * nb:
            break
        agg, nc = dissolve_rank_deficient(agg, nc, B, bs)
        if nc == 0:
            break
        T, Bc = tentative(agg, nc, B, bs)
        P = (T - lv.omega * (Dinv @ (A @ T))).tocsr()
        lv.agg, lv.P = agg, P
        A = (P.T @ A @ P).tocsr()
        B, bs = Bc, B.shape[1]
        th *= 0.5
    Ac = H.levels[-1].A.toarray()
    if Ac.shape[0] > dense_max:
        raise ValueError("coarsest level too large for the dense solve")
    if pin_last:
        # the null vector (the constant pressure) is carried by the first
        # component of every block on every level (the first column of each
        # aggregate's R has zeros below R_00 > 0), so that component of the
        # last block is pinned
        k = Ac.shape[0] - H.levels[-1].bs
        d = Ac[k, k]
        Ac[k, :] = 0.0
        Ac[:, k] = 0.0
        Ac[k, k] = d
    H.coarse_inv = np.linalg.inv(Ac)
    return H


def chebyshev(lv: Level, b: np.ndarray, x: np.ndarray, degree: int) -> np.ndarray:
    """``degree`` Chebyshev steps for A x = b from x with the block-Jacobi
    residual D^-1 (b - A x) on [lo, hi] = [rho/10, rho]."""
    hi = lv.rho
    lo = hi / 10.0
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho_k = 1.0 / sigma
    d = (lv.Dinv @ (b - lv.A @ x)) / theta
    x = x + d
    for _ in range(degree - 1):
        rho_n = 1.0 / (2.0 * sigma - rho_k)
        d = rho_n * rho_k * d + (2.0 * rho_n / delta) * (lv.Dinv @ (b - lv.A @ x))
        x = x + d
        rho_k = rho_n
    return x


def smooth(H: Hierarchy, lv: Level, b: np.ndarray, x) -> np.ndarray:
    """One smoothing of the cycle; x = None starts from zero."""
    if H.smoother == "chebyshev":
        return chebyshev(lv, b, np.zeros_like(b) if x is None else x, H.degree)
    if x is None:
        return lv.omega * (lv.Dinv @ b)
    return x + lv.omega * (lv.Dinv @ (b - lv.A @ x))


def vcycle(H: Hierarchy, b: np.ndarray, level: int = 0) -> np.ndarray:
    lv = H.levels[level]
    if level == len(H.levels) - 1:
        return H.coarse_inv @ b
    x = smooth(H, lv, b, None)
    x = x + lv.P @ vcycle(H, lv.P.T @ (b - lv.A @ x), level + 1)
    return smooth(H, lv, b, x)


def pcg(S, b, H: Hierarchy, rtol=1e-12, maxit=1000):
    """CG on SPD S preconditioned by one block V-cycle (Hestenes & Stiefel,
    1952); stops on the recurrence residual ||r|| <= rtol ||b||."""
    nb = np.linalg.norm(b)
    x = np.zeros_like(b)
    if nb == 0.0:
        return Result(x, 0, 0.0, True)
    r = b.copy()
    z = vcycle(H, r)
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = S @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= rtol * nb:
            return Result(x, it, np.linalg.norm(b - S @ x) / nb, True)
        z = vcycle(H, r)
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return Result(x, maxit, np.linalg.norm(b - S @ x) / nb, False)


def pressure_modes(sys) -> np.ndarray:
    """Near-null space of S for moment pressure DOFs: the DOFs (eq. presMom,
    (1/|P|) int_P q m_a per cell) of q = 1, x, y, z when the pressure space
    holds linear functions (nq = 4), of q = 1 alone for a P0 pressure.
    Needs the cells of the system (assemble(..., keep_local=True))."""
    from .monomials import eval_mono3, mono3
    if sys.cells is None:
        raise ValueError("pressure_modes needs assemble(..., keep_local=True)")
    nq = sys.spec.nq
    if nq == 1:
        return np.ones((sys.n_p, 1))
    if nq != 4:
        raise NotImplementedError("pressure modes for P_k, k > 1")
    out = np.zeros((sys.n_p, 4))
    for c, cell in enumerate(sys.cells):
        Mq = eval_mono3(mono3(1), cell.qp, cell.centroid, cell.diameter)
        Q = np.column_stack([np.ones(cell.qp.shape[0]), cell.qp])
        out[4 * c:4 * c + 4] = (Mq.T * cell.qw) @ Q / cell.volume
    return out


def flux_modes(sys) -> np.ndarray:
    """Near-null space of A_reg = A + B^T B / gamma for the flux DOFs: the
    DOFs (face moments in the global orientation, interior moments) of the
    three constant vector fields, which are divergence-free.  Needs the cells
    of the system (assemble(..., keep_local=True))."""
    from .element import interpolate
    if sys.cells is None:
        raise ValueError("flux_modes needs assemble(..., keep_local=True)")
    out = np.zeros((sys.n_u, 3))
    for c, cell in enumerate(sys.cells):
        for j in range(3):
            e = np.zeros(3)
            e[j] = 1.0
            out[sys.dofmap[c], j] = interpolate(cell, sys.spec, lambda X, e=e: np.tile(e, (X.shape[0], 1)))
    return out


class CondensedCycle:
    """Approximate inverse of the regularised flux block A_reg by exact
    elimination of the interior DOFs cell by cell (their block of A_reg is
    block diagonal over the cells: an interior DOF couples only to its own
    cell) and one V-cycle of this module's point-block AMG on the remaining
    face system S_f = A_ff - A_fi A_ii^-1 A_if, whose bs x bs blocks are the
    nfd face moments of a face:

        r_f' = r_f - A_fi A_ii^-1 r_i,  x_f = V(S_f) r_f',
        x_i  = A_ii^-1 (r_i - A_if x_f).

    Near-null space of S_f: the face DOFs of the three constant fields
    (``flux_modes``); smoothing: block Chebyshev.  Symmetric positive
    definite whenever the V-cycle is (a block LDL^T form with the exact
    interior blocks)."""

    def __init__(self, sys, A_reg: sp.csr_matrix):
        spec = sys.spec
        if spec.nfd < 3:
            raise NotImplementedError("the face blocks must hold the three constant-field modes (nfd >= 3)")
        nf = sys.n_u - spec.nid * sys.vol.size          # face DOFs come first
        A = A_reg.tocsr()
        F = np.arange(nf)
        I = np.arange(nf, sys.n_u)
        self.nf = nf
        self.Afi = A[F][:, I].tocsr()
        if I.size:
            nid = spec.nid
            Aii = A[I][:, I].tocsr()
            blocks = [sp.csr_matrix(np.linalg.inv(Aii[nid * c:nid * (c + 1), nid * c:nid * (c + 1)].toarray()))
                      for c in range(I.size // nid)]
            self.Aii_inv = sp.block_diag(blocks, format="csr")
            self.Sf = (A[F][:, F] - self.Afi @ self.Aii_inv @ self.Afi.T).tocsr()
        else:
            self.Aii_inv = None
            self.Sf = A
        self.H = setup(self.Sf, spec.nfd, flux_modes(sys)[:nf], smoother="chebyshev")

    def __call__(self, r: np.ndarray) -> np.ndarray:
        rf, ri = r[:self.nf], r[self.nf:]
        if self.Aii_inv is None:
            return vcycle(self.H, rf)
        xf = vcycle(self.H, rf - self.Afi @ (self.Aii_inv @ ri))
        return np.concatenate([xf, self.Aii_inv @ (ri - self.Afi.T @ xf)])
