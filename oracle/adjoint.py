"""Gradient of a misfit with respect to per-cell log-permeability (oracle).

With theta_P = log K_P the flux mass matrix is M = sum_P nu_P Mhat_P,
nu_P = exp(-theta_P) (eq. bilin_form with nu = K^{-1}), so
dM/dtheta_P = -M_P (the local matrix of P, scattered).  For
A(theta) x = b with x = (u, p~), p~ = -p, and a loss L(u, p):

    A lambda = dL/dx              (A is symmetric)
    dL/dtheta_P = -lambda^T (dA/dtheta_P) x = lambda_{u,P}^T M_P u_P,

where lambda_{u,P}, u_P are the cell's local flux DOFs and
dL/dp~ = -dL/dp.  Everything here uses the oracle's direct solves.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .assemble import assemble


def gradient_logK(mesh, spec, theta, f, gD, dL_dx, processes=1, solver="direct", rtol=1e-14):
    """(u, p, grad) for the loss whose derivative w.r.t. (u, p) is given by the
    callable dL_dx(u, p) -> (dL/du, dL/dp).  processes: as for assemble().
    solver='direct' factorises A (SuperLU); solver='krylov' solves both
    systems by FGMRES(30) with the block upper-triangular preconditioner and
    an exact (factorised) S to relative residual rtol, for meshes whose
    saddle system SuperLU cannot factorise quickly."""
    nu = np.exp(-np.asarray(theta, dtype=np.float64))
    sys = assemble(mesh, spec, nu, f=f, gD=gD, keep_local=True, processes=processes)
    A = sys.saddle().tocsc()
    if solver == "direct":
        lu = spla.splu(A)
        solve = lu.solve
    elif solver == "krylov":
        from .solvers import BlockPreconditioner, fgmres
        P = BlockPreconditioner(sys, kind="tri", inner="exact")

        def solve(b):
            res = fgmres(A, b, P, restart=30, rtol=rtol, maxit=20000)
            if not res.converged:
                raise RuntimeError(f"oracle FGMRES stopped at relres {res.relres:.2e}")
            return res.x
    else:
        raise ValueError(solver)
    x = solve(sys.rhs())
    u, p = x[:sys.n_u], -x[sys.n_u:]
    gu, gp = dL_dx(u, p)
    lam = solve(np.concatenate([gu, -gp]))     # A^T = A
    lu_u = lam[:sys.n_u]
    grad = np.array([lu_u[dm] @ loc["M"] @ u[dm] for dm, loc in zip(sys.dofmap, sys.local)])
    return u, p, grad


def solve_u_p(mesh, spec, theta, f, gD):
    nu = np.exp(-np.asarray(theta, dtype=np.float64))
    sys = assemble(mesh, spec, nu, f=f, gD=gD)
    x = spla.spsolve(sys.saddle().tocsc(), sys.rhs())
    return x[:sys.n_u], -x[sys.n_u:]
