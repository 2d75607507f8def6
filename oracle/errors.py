"""Error indicators of the paper's convergence test (Sec. 4.4, eq. meshSize and
the indicators e_v, e_q), oracle version.

e_v = sqrt(sum_P ||v - Pi^0_k u_h||^2_{0,P}) / ||v||_{0,Omega}
e_q = sqrt(sum_P ||q - q_h||^2_{0,P}) / ||q||_{0,Omega}
h   = mean of the cell diameters h_P.
"""

from __future__ import annotations

import numpy as np

from .element import local_system
from .monomials import eval_mono3, mono3


def mesh_size(cells) -> float:
    return float(np.mean([c.diameter for c in cells]))


def indicators(sys, cells, dofmaps, u_h, p_h, v_exact, q_exact, nu_cell):
    """Returns (e_v, e_q).  Pressure DOFs are moments (eq. presMom)."""
    spec = sys.spec
    ev2 = en2 = eq2 = eqn2 = 0.0
    qal = mono3(spec.kq)
    for c, cell in enumerate(cells):
        loc = local_system(cell, spec, float(nu_cell[c]), details=True)
        coef = loc["Pi"] @ u_h[dofmaps[c]]            # Pi^0_k u_h in [M_kp]^3
        palph = mono3(spec.kp)
        Mp = eval_mono3(palph, cell.qp, cell.centroid, cell.diameter)
        npal = len(palph)
        uh = np.stack([Mp @ coef[i * npal:(i + 1) * npal] for i in range(3)], 1)
        V = v_exact(cell.qp)
        ev2 += np.sum(cell.qw * np.sum((V - uh) ** 2, 1))
        en2 += np.sum(cell.qw * np.sum(V ** 2, 1))
        # pressure: moments -> coefficients c = |P| Hq^{-1} mom
        mom = p_h[spec.nq * c:spec.nq * (c + 1)]
        cq = np.linalg.solve(loc["Hq"], cell.volume * mom)
        Mq = eval_mono3(qal, cell.qp, cell.centroid, cell.diameter)
        qh = Mq @ cq
        Q = q_exact(cell.qp)
        eq2 += np.sum(cell.qw * (Q - qh) ** 2)
        eqn2 += np.sum(cell.qw * Q ** 2)
    return np.sqrt(ev2 / en2), np.sqrt(eq2 / eqn2)
