"""Local mixed virtual element matrices (oracle), paper Sec. 4.1-4.3.

For a polyhedron P and an element of the family, this computes, in the
paper's order:

1. the face normal traces v.n_f in P_kf(f) from the face moments by the face
   Gram solve (Sec. 4.1, first bullet);
2. div v in P_kq(P) by integration by parts from face traces and gradient
   moments (Sec. 4.1, second bullet);
3. the L2 projection Pi^0_kp onto [P_kp(P)]^3 through the decomposition of
   each vector monomial (eq. decMonoForProj and Props 2.1-2.4, third bullet);
4. the local forms of Sec. 4.3:
     a_{h,P} -> M_P = nu Pi^T H Pi + nu |P| (I - D Pi)^T (I - D Pi)
                (consistency + the dofi-dofi stabilisation s_P),
     b_{h,P} -> B_P[alpha, j] = int_P div(phi_j) psi_alpha = |P| d_j[alpha]
                with psi_alpha the pressure basis dual to the moments of
                eq. presMom,
     f_{h,P} -> F_P[alpha] = int_P f psi_alpha,
   and the Dirichlet term -int_{dP cap dOmega} g_D (phi_j . n_P).

Elements:
* paper k >= 1 (``paper_element(k)``): face moments against M_k(f)
  (eq. facePoly), gradient moments against M_{k-1} minus constants
  (eq. gradMom), cross moments against M^{G,+}_{k-1} (eq. crossMom),
  pressure P_{k-1}, projection Pi^0_k;
* E0: the lowest-order member built by the same recipe with face moments
  against M_0(f) only, no interior moments, P0 pressure and Pi^0_0.  It is
  not in the paper's stated family (whose k = 0 would ask div v in P_{-1});
  it is the element with one normal-flux DOF per face.

Face DOFs are taken against the face's *global* normal, so a face DOF means
the same thing in both cells sharing the face; sigma_{P,f} = +-1 converts to
the outward normal of P.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .monomials import (mono2, mono3, dim_P2, MG_plus, decompose, eval_mono2,
                        eval_mono3, eval_grad_mono3, mI_cross)
from .quadrature import cross3, dunavant4, radon5


@dataclass(frozen=True)
class ElementSpec:
    name: str
    kf: int          # face moments against M_kf(f)
    kp: int          # projection degree (Pi^0_kp)
    kq: int          # pressure / divergence degree
    k: int           # paper order (interior DOFs use k - 1); 0 for E0
    interior: bool

    @property
    def nfd(self) -> int:
        return dim_P2(self.kf)

    @property
    def grad_dofs(self):
        return [a for a in mono3(self.k - 1) if sum(a) >= 1] if self.interior else []

    @property
    def cross_dofs(self):
        return MG_plus(self.k - 1) if self.interior else []

    @property
    def nid(self) -> int:
        return len(self.grad_dofs) + len(self.cross_dofs)

    @property
    def nq(self) -> int:
        return len(mono3(self.kq))


E0 = ElementSpec("E0", kf=0, kp=0, kq=0, k=0, interior=False)


def paper_element(k: int) -> ElementSpec:
    if k < 1:
        raise ValueError("the paper's family starts at k = 1")
    return ElementSpec(f"k{k}", kf=k, kp=k, kq=k - 1, k=k, interior=True)


def _cell_gram(alphas_a, alphas_b, cell):
    Ma = eval_mono3(alphas_a, cell.qp, cell.centroid, cell.diameter)
    Mb = eval_mono3(alphas_b, cell.qp, cell.centroid, cell.diameter)
    return (cell.qw[:, None] * Ma).T @ Mb


def boundary_rule(spec: ElementSpec) -> str:
    """The fan rule of the boundary data.  The patch test of order k has
    g_D in P_{k+1} and u.n in P_k on a face, times the face monomials of
    degree <= k: degree 2k + 1.  Dunavant's degree-4 rule covers E0 and
    k = 1; k = 2 needs degree 5, Radon's rule (for k >= 3 it is the
    highest order at hand, not exact)."""
    return "radon5" if spec.k >= 2 else "dunavant4"


def local_system(cell, spec: ElementSpec, nu: float, f=None, gD=None, details=False, bface_rule=None):
    """Local matrices of cell P.  Returns dict(M, B, F, g[, details...]).

    Local DOF order: for each face of the cell (in the cell's face order) its
    dim P_kf(f) moments (face multi-indices in mono2 order), then gradient
    moments, then cross moments (M^{G,+}_{k-1} order).
    """
    xP, hP, vol = cell.centroid, cell.diameter, cell.volume
    faces = cell.faces
    nfd = spec.nfd
    betas = mono2(spec.kf)
    gdofs = spec.grad_dofs
    cdofs = spec.cross_dofs
    nF = len(faces)
    n_face = nF * nfd
    n_u = n_face + len(gdofs) + len(cdofs)
    gidx = {a: n_face + i for i, a in enumerate(gdofs)}
    cidx = {m: n_face + len(gdofs) + i for i, m in enumerate(cdofs)}

    test = mono3(spec.kp + 1)                       # test monomials incl. the constant
    tpos = {a: i for i, a in enumerate(test)}

    # (1) face traces; boundary term bnd[t, j] = sum_f int_f (phi_j . n_P) m_t
    bnd = np.zeros((len(test), n_u))
    face_ginv = []
    for i, F in enumerate(faces):
        Mf = eval_mono2(betas, F.qp, F)
        Gf = (F.qw[:, None] * Mf).T @ Mf
        Ginv = np.linalg.inv(Gf)
        face_ginv.append(Ginv)
        Mt = eval_mono3(test, F.qp, xP, hP)
        Jf = (F.qw[:, None] * Mf).T @ Mt            # (nfd, ntest)
        # trace of phi_(f,beta) along n_f: |f| sum_gamma Ginv[gamma, beta] m^f_gamma
        bnd[:, i * nfd:(i + 1) * nfd] = F.sigma * F.area * (Jf.T @ Ginv)

    # (2) divergence coefficients d (nq x n_u): H_kq d = r
    qal = mono3(spec.kq)
    Hq = _cell_gram(qal, qal, cell)

    def grad_integral(t):
        """int_P phi_j . grad m_t for all j (row vector), any |t| >= 1."""
        row = np.zeros(n_u)
        if spec.interior and 1 <= sum(t) <= spec.k - 1:
            row[gidx[t]] = vol / hP                  # a gradient moment DOF (eq. gradMom)
            return row
        return None

    r = np.zeros((len(qal), n_u))
    for a_i, a in enumerate(qal):
        gi = np.zeros(n_u) if sum(a) == 0 else grad_integral(a)
        assert gi is not None, "div test monomials of degree <= k-1 are DOFs"
        r[a_i] = -gi + bnd[tpos[a]]
    d = np.linalg.solve(Hq, r)

    # (3) projection: G[i, j] = int_P phi_j . m_i via eq. decMonoForProj
    vecs, grads, crosses, A, C = decompose(spec.kp, hP)
    assert crosses == cdofs
    Hqt = _cell_gram(qal, grads, cell)               # int m_gamma m_beta
    GI = np.zeros((len(grads), n_u))
    for b_i, b in enumerate(grads):
        gi = grad_integral(b)
        if gi is None:
            # integrate by parts: -int div(phi) m_beta + sum_f int_f (phi . n) m_beta
            gi = -(Hqt[:, b_i] @ d) + bnd[tpos[b]]
        GI[b_i] = gi
    CI = np.zeros((len(crosses), n_u))
    for m_i, m in enumerate(crosses):
        CI[m_i, cidx[m]] = vol                       # a cross moment DOF (eq. crossMom)
    G = A @ GI + C @ CI

    pal = mono3(spec.kp)
    Hp = _cell_gram(pal, pal, cell)
    Hvec = np.kron(np.eye(3), Hp)                    # vecs ordered (component, alpha)
    Pi = np.linalg.solve(Hvec, G)

    # DOFs of the vector monomials: D[j, i] = dof_j(m_i)
    D = np.zeros((n_u, len(vecs)))
    for i, F in enumerate(faces):
        Mf = eval_mono2(betas, F.qp, F)
        Ma = eval_mono3(pal, F.qp, xP, hP)
        Jm = (F.qw[:, None] * Mf).T @ Ma            # (nfd, npal)
        for v_i, (c, a) in enumerate(vecs):
            D[i * nfd:(i + 1) * nfd, v_i] = F.normal[c] * Jm[:, pal.index(a)] / F.area
    if spec.interior:
        Mv = eval_mono3(pal, cell.qp, xP, hP)
        for a in gdofs:
            Ga = eval_grad_mono3([a], cell.qp, xP, hP)[:, 0, :]
            for v_i, (c, al) in enumerate(vecs):
                D[gidx[a], v_i] = hP / vol * np.sum(cell.qw * Mv[:, pal.index(al)] * Ga[:, c])
        for m in cdofs:
            W = mI_cross(m[0], m[1], cell.qp, xP, hP)
            for v_i, (c, al) in enumerate(vecs):
                D[cidx[m], v_i] = np.sum(cell.qw * Mv[:, pal.index(al)] * W[:, c]) / vol

    # (4) local forms
    R = np.eye(n_u) - D @ Pi
    M = nu * (Pi.T @ Hvec @ Pi) + nu * vol * (R.T @ R)
    B = vol * d

    Fv = np.zeros(len(qal))
    if f is not None:
        if spec.kq == 0:
            Fv[0] = vol * float(f(xP[None, :])[0])   # cell load rule: midpoint
        else:
            fm = (cell.qw[:, None] * eval_mono3(qal, cell.qp, xP, hP)).T @ f(cell.qp)
            Fv = vol * np.linalg.solve(Hq, fm)

    g = np.zeros(n_u)
    if gD is not None:
        for i, F in enumerate(faces):
            if F.bc != 1:
                continue
            pts, wts = load_face_points(F, bface_rule or boundary_rule(spec))
            Mf = eval_mono2(betas, pts, F)
            gm = (wts[:, None] * Mf).T @ gD(pts)     # int_f g_D m^f_gamma
            g[i * nfd:(i + 1) * nfd] = -F.sigma * F.area * (face_ginv[i].T @ gm)

    out = dict(M=M, B=B, F=Fv, g=g)
    if details:
        out.update(Pi=Pi, D=D, Hvec=Hvec, d=d, G=G, Hq=Hq, vecs=vecs)
    return out


def load_face_points(F, rule="dunavant4"):
    """Boundary-face load rule on the fan (x_f, v_i, v_{i+1}): Dunavant's
    degree-4 rule, or rule='radon5', Radon's degree-5 rule (boundary_rule
    gives the one of an element)."""
    tri = {"dunavant4": dunavant4, "radon5": radon5}[rule]
    V = F.verts
    m = V.shape[0]
    pts, wts = [], []
    for i in range(m):
        A, B = V[i], V[(i + 1) % m]
        p, w = tri(F.centroid, A, B)
        s = np.sign(np.dot(cross3(A - F.centroid, B - F.centroid), F.normal))
        pts.append(p)
        wts.append(w * s)
    return np.concatenate(pts), np.concatenate(wts)


def interpolate(cell, spec: ElementSpec, v):
    """DOFs of a vector field v (callable (N,3)->(N,3)) in cell P: face moments
    against the global normal, gradient moments, cross moments (eq. facePoly,
    gradMom, crossMom), by exact-integration quadrature."""
    xP, hP, vol = cell.centroid, cell.diameter, cell.volume
    betas = mono2(spec.kf)
    out = []
    for F in cell.faces:
        Mf = eval_mono2(betas, F.qp, F)
        vn = v(F.qp) @ F.normal
        out.append((F.qw * vn) @ Mf / F.area)
    if spec.interior:
        V = v(cell.qp)
        for a in spec.grad_dofs:
            Ga = eval_grad_mono3([a], cell.qp, xP, hP)[:, 0, :]
            out.append(np.array([hP / vol * np.sum(cell.qw * np.sum(V * Ga, 1))]))
        for m in spec.cross_dofs:
            W = mI_cross(m[0], m[1], cell.qp, xP, hP)
            out.append(np.array([np.sum(cell.qw * np.sum(V * W, 1)) / vol]))
    return np.concatenate(out)
