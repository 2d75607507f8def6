"""Solvers for the saddle-point system (oracle).

Paper Sec. 5: the system matrix [A B^T; B -C] (here C = 0, A = M) is solved
by GMRES with a block preconditioner.  Block-Schur (eq. block_schur):
B_1 = diag(A), B_2^{-1} = exact solve with S = B diag(A)^{-1} B^T (the sign of
the paper's S = -C - B diag(A)^{-1} B^T is absorbed by solving for p~ = -p).
This module also holds the two variants the project adds around it: the
same block-diagonal preconditioner inside MINRES (it is SPD, so MINRES
applies), and the block upper-triangular form
    P = [diag(M)  B^T; 0  -S],   P^{-1} r: z_p = -S^{-1} r_p,
                                           z_u = diag(M)^{-1}(r_u - B^T z_p).

Krylov methods, written from their textbook statements:
* preconditioned MINRES: C.C. Paige & M.A. Saunders, SIAM J. Numer. Anal.
  12 (1975); the preconditioned Lanczos form of H. Elman, D. Silvester,
  A. Wathen, "Finite Elements and Fast Iterative Solvers" (2005), Alg. 4.1;
* FGMRES(m): Y. Saad, SIAM J. Sci. Comput. 14 (1993) -- right
  preconditioning, modified Gram-Schmidt Arnoldi, Givens rotations;
* Jacobi-preconditioned CG for S: Hestenes & Stiefel (1952).
All stop on the TRUE relative residual ||b - A x||_2 / ||b||_2.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


@dataclass
class Result:
    x: np.ndarray
    iters: int
    relres: float
    converged: bool
    inner_iters: int = 0


def solve_direct(sys, return_multiplier=False):
    """Direct sparse solve; returns (u, p) with the physical pressure sign
    (and the mean-zero multiplier when asked; 0 without one)."""
    if sys.multiplier:
        A, b = sys.augmented()
        x = spla.spsolve(A.tocsc(), b)
        lam = x[-1]
        x = x[:-1]
    else:
        x = spla.spsolve(sys.saddle().tocsc(), sys.rhs())
        lam = 0.0
    u, p = x[:sys.n_u], -x[sys.n_u:sys.n_u + sys.n_p]
    return (u, p, lam) if return_multiplier else (u, p)


def schur(sys) -> sp.csr_matrix:
    """S = B diag(M)^{-1} B^T over the free flux DOFs (prescribed-flux DOFs
    are eliminated, so their columns of B do not enter)."""
    dinv = 1.0 / sys.M.diagonal()
    B = sys.B
    if sys.fixed is not None and sys.fixed.size:
        keep = np.ones(sys.n_u)
        keep[sys.fixed] = 0.0
        B = B @ sp.diags(keep)
    return (B @ sp.diags(dinv) @ B.T).tocsr()


def pcg(S, b, rtol=1e-12, maxit=10000, x0=None):
    """Jacobi-preconditioned CG on SPD S; stops on ||b - S x|| <= rtol ||b||."""
    dinv = 1.0 / S.diagonal()
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - S @ x
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return Result(np.zeros_like(b), 0, 0.0, True)
    z = dinv * r
    p = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = S @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        if np.linalg.norm(r) <= rtol * nb:
            return Result(x, it, np.linalg.norm(b - S @ x) / nb, True)
        z = dinv * r
        rz_new = r @ z
        p = z + (rz_new / rz) * p
        rz = rz_new
    return Result(x, maxit, np.linalg.norm(b - S @ x) / nb, False)


def mesh_size(sys) -> float:
    """h = (1/N_P) sum_P h_P, the mean cell diameter (Sec. 6, eq. meshSize)."""
    return float(np.mean(sys.diam))


def regularized(sys, gamma: float) -> sp.csr_matrix:
    """A + B^T W^{-1} B with W = gamma I (Block-Reg, Sec. 5) over the free
    flux DOFs: the prescribed-flux DOFs keep a unit row and column, as in the
    eliminated saddle-point matrix."""
    keep = np.ones(sys.n_u)
    if sys.fixed is not None and sys.fixed.size:
        keep[sys.fixed] = 0.0
    K = sp.diags(keep)
    BK = sys.B @ K
    return (K @ sys.M @ K + (1.0 / gamma) * (BK.T @ BK) + sp.diags(1.0 - keep)).tocsr()


class BlockPreconditioner:
    """Block-diagonal (kind='diag') or block upper-triangular (kind='tri')
    preconditioner with diag(M) for the flux block and S = B diag(M)^{-1} B^T
    for the pressure block.  inner='exact' factorises S (the paper's choice,
    with MUMPS there and SuperLU here); inner='pcg' uses Jacobi-PCG to
    inner_rtol; inner='amg' uses CG preconditioned by one V-cycle of the
    smoothed-aggregation AMG of oracle/amg.py to inner_rtol; inner='block-amg'
    the same with the point-block AMG of oracle/block_amg.py (a cell's
    pressure moments kept together, near-null space the moments of 1, x, y,
    z; needs assemble(..., keep_local=True)).

    kind='reg' is the paper's Block-Reg (Sec. 5): block-diagonal with one
    V-cycle of the smoothed-aggregation AMG of A + B^T W^{-1} B (Chebyshev
    smoothing, as in the GAMG preconditioner the paper names; with
    reg_smoother='edge-schwarz' the edge-patch Schwarz smoothing of
    oracle/schwarz.py on the finest level, which needs the mesh; with
    reg_smoother='block-chebyshev' (k = 1) the point-block AMG of
    oracle/block_amg.py on 3 x 3 blocks with the constant fields as
    near-null space; with reg_smoother='condensed-block' the interior DOFs
    eliminated cell by cell and that AMG on the face system,
    block_amg.CondensedCycle) for the flux
    block and W^{-1} = I / gamma for the pressure block; gamma defaults to
    h^2, h the mean cell diameter (the paper's choice)."""

    def __init__(self, sys, kind="diag", inner="exact", inner_rtol=1e-12, inner_maxit=10000, gamma=None,
                 reg_smoother="chebyshev", mesh=None):
        self.n_u = sys.n_u
        self.kind = kind
        self.inner_iters = 0
        if kind == "reg":
            from . import amg
            self.amg = amg
            self.gamma = mesh_size(sys) ** 2 if gamma is None else float(gamma)
            self.A_reg = regularized(sys, self.gamma)
            if reg_smoother == "chebyshev":
                H = amg.setup(self.A_reg, smoother="chebyshev")
                self.cycle_reg = lambda r: amg.vcycle(H, r)
                self.H_reg = H
            elif reg_smoother == "block-chebyshev":
                from . import block_amg
                if not (sys.spec.nfd == sys.spec.nid == 3):
                    raise NotImplementedError("3 x 3 flux blocks need the paper's k = 1 element")
                Hb = block_amg.setup(self.A_reg, 3, block_amg.flux_modes(sys), smoother="chebyshev")
                self.cycle_reg = lambda r: block_amg.vcycle(Hb, r)
                self.H_reg = Hb
            elif reg_smoother == "condensed-block":
                from . import block_amg
                self.cycle_reg = block_amg.CondensedCycle(sys, self.A_reg)
            elif reg_smoother == "edge-schwarz":
                from . import schwarz
                if mesh is None:
                    raise ValueError("the edge-patch smoother needs the mesh")
                self.cycle_reg = schwarz.setup(self.A_reg, schwarz.edge_patches(mesh, sys.spec))
            else:
                raise ValueError(reg_smoother)
            return
        self.B = sys.B
        self.dM = sys.M.diagonal().copy()
        self.S = schur(sys)
        self.inner = inner
        self.inner_rtol = inner_rtol
        self.inner_maxit = inner_maxit
        self.fixed = sys.fixed if sys.fixed is not None else np.zeros(0, dtype=np.int64)
        if self.fixed.size:
            self.B = (self.B @ sp.diags(np.where(np.isin(np.arange(sys.n_u), self.fixed), 0.0, 1.0))).tocsr()
            self.dM[self.fixed] = 1.0
        self.multiplier = sys.multiplier
        if sys.multiplier:
            self.e = sys.null_vec
        if inner == "exact":
            if sys.multiplier:
                # singular S (constants): factorise [[S, c], [c^T, 0]]
                c = sp.csr_matrix(sys.cvec[:, None])
                self.lu = spla.splu(sp.bmat([[self.S, c], [c.T, None]], format="csc"))
            else:
                self.lu = spla.splu(self.S.tocsc())
        elif inner == "amg":
            from . import amg
            self.amg = amg
            if sys.multiplier and sys.n_p != sys.vol.size:
                raise NotImplementedError("AMG with the multiplier needs one pressure DOF per cell")
            self.H = amg.setup(self.S, pin_last=sys.multiplier)
        elif inner == "block-amg":
            from . import block_amg
            self.bamg = block_amg
            self.H = block_amg.setup(self.S, sys.spec.nq, block_amg.pressure_modes(sys), pin_last=sys.multiplier)

    def solve_S(self, r):
        if self.multiplier:
            # the consistent part (range of S = orthogonal complement of e)
            r = r - (self.e @ r) / (self.e @ self.e) * self.e
        if self.inner == "exact":
            if self.multiplier:
                return self.lu.solve(np.concatenate([r, [0.0]]))[:-1]
            return self.lu.solve(r)
        if self.inner == "amg":
            res = self.amg.amg_pcg(self.S, r, self.H, self.inner_rtol, self.inner_maxit)
        elif self.inner == "block-amg":
            res = self.bamg.pcg(self.S, r, self.H, self.inner_rtol, self.inner_maxit)
        else:
            res = pcg(self.S, r, self.inner_rtol, self.inner_maxit)
        self.inner_iters += res.iters
        return res.x

    def __call__(self, r):
        ru, rp = r[:self.n_u], r[self.n_u:]
        if self.kind == "reg":
            return np.concatenate([self.cycle_reg(ru), rp / self.gamma])
        if self.kind == "diag":
            return np.concatenate([ru / self.dM, self.solve_S(rp)])
        zp = -self.solve_S(rp)
        zu = (ru - self.B.T @ zp) / self.dM
        return np.concatenate([zu, zp])


def minres(A, b, Pinv, rtol=1e-12, maxit=5000):
    """Preconditioned MINRES for symmetric A with SPD preconditioner Pinv."""
    n = b.size
    nb = np.linalg.norm(b)
    x = np.zeros(n)
    if nb == 0.0:
        return Result(x, 0, 0.0, True)
    v_old = np.zeros(n)
    v = b.copy()
    z = Pinv(v)
    gamma = np.sqrt(v @ z)
    gamma_old = 1.0
    eta = gamma
    c_old, c = 1.0, 1.0
    s_old, s = 0.0, 0.0
    w_old = np.zeros(n)
    w = np.zeros(n)
    for it in range(1, maxit + 1):
        z = z / gamma
        Az = A @ z
        delta = Az @ z
        v_new = Az - (delta / gamma) * v - (gamma / gamma_old) * v_old
        z_new = Pinv(v_new)
        gamma_new = np.sqrt(max(v_new @ z_new, 0.0))
        a0 = c * delta - c_old * s * gamma
        a1 = np.hypot(a0, gamma_new)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_new, s_new = a0 / a1, gamma_new / a1
        w_new = (z - a3 * w_old - a2 * w) / a1
        x = x + c_new * eta * w_new
        eta = -s_new * eta
        rel = np.linalg.norm(b - A @ x) / nb
        if rel <= rtol:
            return Result(x, it, rel, True)
        if gamma_new == 0.0:
            return Result(x, it, rel, False)
        v_old, v = v, v_new
        z = z_new
        gamma_old, gamma = gamma, gamma_new
        c_old, c = c, c_new
        s_old, s = s, s_new
        w_old, w = w, w_new
    return Result(x, maxit, np.linalg.norm(b - A @ x) / nb, False)


def fgmres(A, b, Pinv, restart=30, rtol=1e-12, maxit=5000):
    """Restarted flexible GMRES with right preconditioning, x0 = 0."""
    n = b.size
    nb = np.linalg.norm(b)
    x = np.zeros(n)
    if nb == 0.0:
        return Result(x, 0, 0.0, True)
    total = 0
    while total < maxit:
        r = b - A @ x
        beta = np.linalg.norm(r)
        if beta <= rtol * nb:
            return Result(x, total, beta / nb, True)
        m = restart
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        gvec = np.zeros(m + 1)
        gvec[0] = beta
        V[0] = r / beta
        j_done = 0
        for j in range(m):
            Z[j] = Pinv(V[j])
            w = A @ Z[j]
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            gvec[j + 1] = -sn[j] * gvec[j]
            gvec[j] = cs[j] * gvec[j]
            total += 1
            j_done = j + 1
            if abs(gvec[j + 1]) <= rtol * nb or total >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:j_done, :j_done]), gvec[:j_done])
        x = x + Z[:j_done].T @ y
        rel = np.linalg.norm(b - A @ x) / nb
        if rel <= rtol:
            return Result(x, total, rel, True)
    return Result(x, total, np.linalg.norm(b - A @ x) / nb, False)


def solve_krylov(sys, method="minres", kind="diag", inner="exact", rtol=1e-12,
                 inner_rtol=1e-12, restart=30, maxit=5000, gamma=None, reg_smoother="chebyshev", mesh=None):
    """Preconditioned Krylov solve; returns (u, p, Result) with physical p.
    With the mean-zero multiplier the pressure equations are made consistent
    first (F - c lambda with lambda = sum F / sum c, the multiplier's value),
    the singular system is solved and p is shifted to mean zero."""
    A = sys.saddle()
    b = sys.rhs()
    if sys.multiplier:
        # e^T (B u + c lambda) = e^T F with B^T e = 0
        e, c = sys.null_vec, sys.cvec
        lam = (e @ b[sys.n_u:]) / (e @ c)
        b[sys.n_u:] -= c * lam
    P = BlockPreconditioner(sys, kind=kind, inner=inner, inner_rtol=inner_rtol, gamma=gamma,
                            reg_smoother=reg_smoother, mesh=mesh)
    if method == "minres":
        if kind not in ("diag", "reg"):
            raise ValueError("MINRES needs an SPD block-diagonal preconditioner")
        res = minres(A, b, P, rtol=rtol, maxit=maxit)
    elif method == "fgmres":
        res = fgmres(A, b, P, restart=restart, rtol=rtol, maxit=maxit)
    else:
        raise ValueError(method)
    res.inner_iters = P.inner_iters
    u, pt = res.x[:sys.n_u], res.x[sys.n_u:]
    if sys.multiplier:
        e, c = sys.null_vec, sys.cvec
        pt = pt - (c @ pt) / (c @ e) * e
    return u, -pt, res
