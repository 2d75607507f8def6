"""Smoothed-aggregation algebraic multigrid for the Schur block S (oracle).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper solves S exactly (MUMPS) inside Block-Schur and uses PETSc's GAMG,
a smoothed-aggregation AMG, for the velocity block of Block-Reg (Sec. 5).
The library offers an AMG-preconditioned CG as its inner solver for S; this
module defines that AMG, written from the published method:

* smoothed aggregation: P. Vanek, J. Mandel, M. Brezina, "Algebraic
  multigrid by smoothed aggregation for second and fourth order elliptic
  problems", Computing 56 (1996): strength |a_ij| >= theta sqrt(a_ii a_jj),
  piecewise-constant tentative prolongator T, P = (I - omega D^-1 A) T,
  Galerkin coarse operator P^T A P, theta halved on every coarser level;
* aggregation by a distance-2 maximal independent set of the strength graph
  (N. Bell, S. Dalton, L. N. Olson, SIAM J. Sci. Comput. 34 (2012)).  The
  set is defined here as the greedy one on the square of the graph, taken in
  decreasing order of a fixed key per node; parallel rounds in which a node
  joins when its key is the largest among the undecided nodes within
  distance 2 compute the same set.

Exact rules (the integer decisions -- strength, roots, aggregates -- are
reproduced bit for bit by the library):

* strong(i, j): j != i and |a_ij| >= theta * sqrt(a_ii * a_jj), with a_ij
  read from row i; the neighbours of i are the strong entries of row i.
* key(i) = ((splitmix64(i) >> 34) << 32) | i  (unique, 62 bits), splitmix64
  the output function of G. Steele, D. Lea, C. Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014.
* roots: greedy distance-2 independent set in decreasing key order; root
  aggregates are numbered in increasing node index.
* pass 1: a non-root node joins the smallest root aggregate among its
  strong neighbours that are roots;
* pass 2: a node still free joins the smallest aggregate among its strong
  neighbours placed in pass 1;
* isolated node: a row without strong entries.  It stays out of the coarse
  space (its row of P is zero); Jacobi smoothing handles it.
* pass 3: a non-isolated node still free becomes a singleton aggregate,
  numbered after the root aggregates in increasing node index.  Root
  aggregates count only non-isolated roots.
* prolongator smoothing uses the filtered matrix A^F (the diagonal and the
  strong entries of A; weak entries dropped):
  P = T - omega_F D^-1 A^F T, omega_F = 4 / (3 rho_F),
  rho_F = max_i sum_j |a^F_ij| / a_ii.
* Jacobi weight omega = 4 / (3 rho), rho = max_i sum_j |a_ij| / a_ii
  (Gershgorin bound of rho(D^-1 A)).
* coarsening stops when a level has at most ``coarse_max`` rows, when the
  next level would keep more than 4/5 of the rows or none, or at
  ``max_levels``; the coarsest level is solved exactly (dense inverse) when
  it has at most ``dense_max`` rows, else by ``coarse_sweeps`` damped-Jacobi
  sweeps from zero.

Cycle (symmetric, so it preconditions CG): V(1,1) with damped Jacobi,
    x = w D^-1 b;  x += P V(P^T (b - A x));  x += w D^-1 (b - A x),
or (smoother='chebyshev', the default smoother of PETSc's GAMG, which the
paper uses for Block-Reg) the same V-cycle with two steps of Chebyshev
acceleration of the Jacobi iteration before and after the coarse
correction: Y. Saad, "Iterative Methods for Sparse Linear Systems", 2nd ed.
(2003), Algorithm 12.1, applied to D^-1 A on the interval [rho/10, rho],
rho the Gershgorin bound above (an upper bound of the spectrum of D^-1 A,
so every eigenvalue's error factor has modulus below one and the cycle stays
symmetric positive definite).
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .solvers import Result

MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """Output function of SplitMix64 applied to the counter value x."""
    z = (x + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def node_key(i: int) -> int:
    return ((splitmix64(i) >> 34) << 32) | i


def strength(A: sp.csr_matrix, theta: float):
    """Row-wise strong neighbour lists (CSR pointer and indices)."""
    A = A.tocsr()
    d = A.diagonal()
    ptr = [0]
    idx = []
    for i in range(A.shape[0]):
        for k in range(A.indptr[i], A.indptr[i + 1]):
            j = int(A.indices[k])
            if j != i and abs(A.data[k]) >= theta * np.sqrt(d[i] * d[j]):
                idx.append(j)
        ptr.append(len(idx))
    return np.array(ptr, dtype=np.int64), np.array(idx, dtype=np.int64)


def mis2(n: int, ptr, idx):
    """Greedy distance-2 independent set in decreasing key order."""
    order = sorted(range(n), key=node_key, reverse=True)
    blocked = np.zeros(n, dtype=bool)
    root = np.zeros(n, dtype=bool)
    for i in order:
        if blocked[i]:
            continue
        root[i] = True
        blocked[i] = True
        for j in idx[ptr[i]:ptr[i + 1]]:
            blocked[j] = True
            for k in idx[ptr[j]:ptr[j + 1]]:
                blocked[k] = True
    return root


def aggregate(n: int, ptr, idx):
    """Aggregate id per node (-1 for isolated nodes) and the number of
    aggregates."""
    root = mis2(n, ptr, idx)
    iso = np.diff(ptr) == 0
    croot = root & ~iso
    rid = np.cumsum(croot) - 1
    agg1 = np.full(n, -1, dtype=np.int64)
    for i in range(n):
        if iso[i]:
            continue
        if croot[i]:
            agg1[i] = rid[i]
            continue
        best = -1
        for j in idx[ptr[i]:ptr[i + 1]]:
            if croot[j] and (best < 0 or rid[j] < best):
                best = rid[j]
        agg1[i] = best
    agg = agg1.copy()
    for i in range(n):
        if agg1[i] >= 0 or iso[i]:
            continue
        best = -1
        for j in idx[ptr[i]:ptr[i + 1]]:
            if agg1[j] >= 0 and (best < 0 or agg1[j] < best):
                best = agg1[j]
        agg[i] = best
    nroot = int(croot.sum())
    free = np.nonzero((agg < 0) & ~iso)[0]
    agg[free] = nroot + np.arange(free.size)
    return agg, nroot + free.size


def gershgorin_rho(A: sp.csr_matrix) -> float:
    """max_i sum_j |a_ij| / a_ii."""
    A = A.tocsr()
    rows = np.asarray(abs(A).sum(axis=1)).ravel()
    return float((rows / A.diagonal()).max())


def filtered(A: sp.csr_matrix, ptr, idx) -> sp.csr_matrix:
    """The diagonal and the strong entries of A (weak entries dropped)."""
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(ptr))
    St = sp.csr_matrix((np.ones(idx.size), (rows, idx)), shape=A.shape)
    return (A.multiply(St) + sp.diags(A.diagonal())).tocsr()


@dataclass
class Level:
    A: sp.csr_matrix
    dinv: np.ndarray
    omega: float
    rho: float = 0.0                   # Gershgorin bound of rho(D^-1 A)
    agg: np.ndarray = None
    P: sp.csr_matrix = None


@dataclass
class Hierarchy:
    levels: list = field(default_factory=list)
    coarse_inv: np.ndarray = None      # dense inverse of the coarsest A, or None
    coarse_sweeps: int = 0             # else: damped-Jacobi sweeps from zero
    smoother: str = "jacobi"           # 'jacobi' (one step) or 'chebyshev'
    degree: int = 2                    # Chebyshev steps per smoothing

    @property
    def sizes(self):
        return [lv.A.shape[0] for lv in self.levels]

    def operator_complexity(self):
        return sum(lv.A.nnz for lv in self.levels) / self.levels[0].A.nnz


def setup(A: sp.csr_matrix, theta: float = 0.08, coarse_max: int = 64, max_levels: int = 12,
          dense_max: int = 512, coarse_sweeps: int = 4, pin_last: bool = False,
          smoother: str = "jacobi", degree: int = 2) -> Hierarchy:
    """pin_last: A is singular with the constants as null space (flux data
    on the whole boundary); the coarsest matrix then keeps the diagonal of its
    last row and column and drops their other entries before inversion,
    which leaves a symmetric positive definite cycle.  smoother / degree:
    the cycle's smoother (module docstring); the hierarchy does not depend
    on it."""
    if smoother not in ("jacobi", "chebyshev"):
        raise ValueError(smoother)
    H = Hierarchy(smoother=smoother, degree=degree)
    A = A.tocsr()
    th = theta
    while True:
        rho = gershgorin_rho(A)
        lv = Level(A=A, dinv=1.0 / A.diagonal(), omega=4.0 / (3.0 * rho), rho=rho)
        H.levels.append(lv)
        n = A.shape[0]
        if n <= coarse_max or len(H.levels) == max_levels:
            break
        ptr, idx = strength(A, th)
        agg, nc = aggregate(n, ptr, idx)
        if nc == 0 or 5 * nc > 4 * n:
            break
        AF = filtered(A, ptr, idx)
        omega_f = 4.0 / (3.0 * gershgorin_rho(AF))
        m = agg >= 0
        T = sp.csr_matrix((np.ones(int(m.sum())), (np.arange(n)[m], agg[m])), shape=(n, nc))
        P = (T - omega_f * sp.diags(lv.dinv) @ AF @ T).tocsr()
        lv.agg, lv.P = agg, P
        A = (P.T @ A @ P).tocsr()
        th *= 0.5
    if H.levels[-1].A.shape[0] <= dense_max:
        Ac = H.levels[-1].A.toarray()
        if pin_last:
            d = Ac[-1, -1]
            Ac[-1, :] = 0.0
            Ac[:, -1] = 0.0
            Ac[-1, -1] = d
        H.coarse_inv = np.linalg.inv(Ac)
    else:
        H.coarse_sweeps = coarse_sweeps
    return H


def coarse_solve(H: Hierarchy, b: np.ndarray) -> np.ndarray:
    if H.coarse_inv is not None:
        return H.coarse_inv @ b
    lv = H.levels[-1]
    x = lv.omega * lv.dinv * b
    for _ in range(H.coarse_sweeps - 1):
        x = x + lv.omega * lv.dinv * (b - lv.A @ x)
    return x


def chebyshev(lv: Level, b: np.ndarray, x: np.ndarray, degree: int) -> np.ndarray:
    """degree steps of Chebyshev acceleration of the Jacobi iteration for
    A x = b from x (Saad 2003, Algorithm 12.1 with residual D^-1 (b - A x)),
    on the interval [lo, hi] = [rho/10, rho]."""
    hi = lv.rho
    lo = hi / 10.0
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    rho_k = 1.0 / sigma
    d = lv.dinv * (b - lv.A @ x) / theta
    x = x + d
    for _ in range(degree - 1):
        rho_n = 1.0 / (2.0 * sigma - rho_k)
        d = rho_n * rho_k * d + (2.0 * rho_n / delta) * (lv.dinv * (b - lv.A @ x))
        x = x + d
        rho_k = rho_n
    return x


def smooth(H: Hierarchy, lv: Level, b: np.ndarray, x) -> np.ndarray:
    """One smoothing of the cycle; x = None starts from zero."""
    if H.smoother == "chebyshev":
        return chebyshev(lv, b, np.zeros_like(b) if x is None else x, H.degree)
    if x is None:
        return lv.omega * lv.dinv * b
    return x + lv.omega * lv.dinv * (b - lv.A @ x)


def vcycle(H: Hierarchy, b: np.ndarray, level: int = 0) -> np.ndarray:
    lv = H.levels[level]
    if level == len(H.levels) - 1:
        return coarse_solve(H, b)
    x = smooth(H, lv, b, None)
    r = b - lv.A @ x
    x = x + lv.P @ vcycle(H, lv.P.T @ r, level + 1)
    return smooth(H, lv, b, x)


def amg_pcg(S, b, H: Hierarchy, rtol=1e-12, maxit=1000):
    """CG on SPD S preconditioned by one V-cycle (Hestenes & Stiefel, 1952);
    stops on the recurrence residual ||r|| <= rtol ||b||."""
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
