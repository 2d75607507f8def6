"""Scaled monomials and the vector-monomial decomposition (oracle).

Paper Sec. 2: scaled monomials m_alpha = ((x - x_P)/h_P)^alpha (eq. monoBasis),
face monomials m^f_beta in the face frame, vector monomials [M_k(P)]^3, the
decomposition [P_k]^3 = G_k (+) G_k^+ (eq. spaceDec, decomp) with the closed
forms of Props 2.1-2.3 (eq. decForX and its y/z analogues), the rewriting of
Prop 2.4, the sets N_k (eq. NDef) and M^{G,+}_k (Sec. 2.2).

Reading of eq. NDef: N_k must contain the constant (0 <= |alpha| <= k with
alpha_1 = 0).  With 0 < |alpha| the dimension count of Sec. 2.2 (and every
DOF count of Tables 1-6) fails: dim M^{G,+}_0 would be 2, not 3.

Ordering: multi-indices by total degree, then by descending alpha_1, then
descending alpha_2 -- for degree <= 1: (000),(100),(010),(001).  Face
multi-indices likewise: (00),(10),(01),(20),(11),(02),...
"""

from __future__ import annotations

import numpy as np


def mono3(k: int):
    """3D multi-indices with 0 <= |alpha| <= k."""
    out = []
    for d in range(k + 1):
        for a1 in range(d, -1, -1):
            for a2 in range(d - a1, -1, -1):
                out.append((a1, a2, d - a1 - a2))
    return out


def mono2(k: int):
    out = []
    for d in range(k + 1):
        for b1 in range(d, -1, -1):
            out.append((b1, d - b1))
    return out


def dim_P3(k: int) -> int:
    return 0 if k < 0 else (k + 1) * (k + 2) * (k + 3) // 6


def dim_P2(k: int) -> int:
    return 0 if k < 0 else (k + 1) * (k + 2) // 2


def N_set(k: int):
    """eq. NDef with the constant included: alpha_1 = 0, |alpha| <= k."""
    return [a for a in mono3(k) if a[0] == 0]


def MG_plus(k: int):
    """M^{G,+}_k(P) as a list of (component, alpha): x-component over N_k,
    y- and z-components over all of M_k (Sec. 2.2)."""
    if k < 0:
        return []
    return ([(0, a) for a in N_set(k)] + [(1, a) for a in mono3(k)] + [(2, a) for a in mono3(k)])


def eval_mono3(alphas, X, xP, hP):
    """(N, len(alphas)) values of m_alpha at points X."""
    Y = (X - xP[None, :]) / hP
    out = np.empty((X.shape[0], len(alphas)))
    for j, a in enumerate(alphas):
        out[:, j] = Y[:, 0] ** a[0] * Y[:, 1] ** a[1] * Y[:, 2] ** a[2]
    return out


def eval_grad_mono3(alphas, X, xP, hP):
    """(N, len(alphas), 3) values of grad m_alpha."""
    Y = (X - xP[None, :]) / hP
    out = np.zeros((X.shape[0], len(alphas), 3))
    for j, a in enumerate(alphas):
        for c in range(3):
            if a[c] == 0:
                continue
            e = list(a)
            e[c] -= 1
            out[:, j, c] = a[c] * Y[:, 0] ** e[0] * Y[:, 1] ** e[1] * Y[:, 2] ** e[2] / hP
    return out


def eval_mono2(betas, X, face):
    """Face scaled monomials m^f_beta = ((x~ - x~_f)/h_f)^beta in the face frame."""
    D = X - face.centroid[None, :]
    s = D @ face.t1 / face.diameter
    t = D @ face.t2 / face.diameter
    out = np.empty((X.shape[0], len(betas)))
    for j, b in enumerate(betas):
        out[:, j] = s ** b[0] * t ** b[1]
    return out


def mI_cross(comp: int, alpha, X, xP, hP):
    """(N, 3) values of m_I ^ (e_comp m_alpha), m_I = (x - x_P)/h_P."""
    Y = (X - xP[None, :]) / hP
    m = Y[:, 0] ** alpha[0] * Y[:, 1] ** alpha[1] * Y[:, 2] ** alpha[2]
    e = np.zeros((X.shape[0], 3))
    e[:, comp] = m
    return np.cross(Y, e)


def decompose(kp: int, hP: float):
    """Decomposition of every vector monomial e_c m_alpha, |alpha| <= kp.

    Returns (vecs, grads, crosses, A, C):
      vecs    list of (c, alpha)                    the vector monomials [M_kp]^3
      grads   list of beta, 0 < |beta| <= kp + 1    (basis of G_kp, eq. GBasis)
      crosses M^{G,+}_{kp-1} as (comp, gamma)
      A       (n_vec, n_grad) coefficients of grad m_beta
      C       (n_vec, n_cross) coefficients of m_I ^ (e_comp m_gamma)
    following Props 2.1-2.3, with any x-component cross term (m_gamma, 0, 0),
    gamma_1 > 0, rewritten by Prop 2.4.
    """
    alphas = mono3(kp)
    vecs = [(c, a) for c in range(3) for a in alphas]
    grads = [b for b in mono3(kp + 1) if sum(b) > 0]
    crosses = MG_plus(kp - 1)
    gi = {b: i for i, b in enumerate(grads)}
    ci = {m: i for i, m in enumerate(crosses)}
    A = np.zeros((len(vecs), len(grads)))
    C = np.zeros((len(vecs), len(crosses)))

    def add_cross(row, comp, gamma, coef):
        if coef == 0.0:
            return
        if any(g < 0 for g in gamma):
            raise AssertionError("negative index with non-zero coefficient")
        if comp == 0 and gamma[0] > 0:
            # Prop 2.4: m_I ^ (m_g,0,0) = -m_I ^ (0,m_b,0) - m_I ^ (0,0,m_c)
            b = (gamma[0] - 1, gamma[1] + 1, gamma[2])
            cc = (gamma[0] - 1, gamma[1], gamma[2] + 1)
            C[row, ci[(1, b)]] -= coef
            C[row, ci[(2, cc)]] -= coef
        else:
            C[row, ci[(comp, gamma)]] += coef

    for r, (c, a) in enumerate(vecs):
        s = sum(a) + 1.0
        beta = list(a)
        beta[c] += 1
        A[r, gi[tuple(beta)]] += hP / s
        a1, a2, a3 = a
        if c == 0:     # Prop 2.1
            add_cross(r, 1, (a1, a2, a3 - 1), -a3 / s)
            add_cross(r, 2, (a1, a2 - 1, a3), a2 / s)
        elif c == 1:   # Prop 2.2
            add_cross(r, 0, (a1, a2, a3 - 1), a3 / s)
            add_cross(r, 2, (a1 - 1, a2, a3), -a1 / s)
        else:          # Prop 2.3
            add_cross(r, 1, (a1 - 1, a2, a3), a1 / s)
            add_cross(r, 0, (a1, a2 - 1, a3), -a2 / s)
    return vecs, grads, crosses, A, C
