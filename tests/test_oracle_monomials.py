"""Pins for oracle/monomials.py against the paper's Sec. 2 statements."""

import numpy as np
import pytest

from oracle.monomials import (MG_plus, decompose, dim_P3, eval_grad_mono3, eval_mono3,
                              mI_cross, mono3)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 4])
def test_decomposition_reproduces_vector_monomials(k):
    """eq. decomp: every e_c m_alpha equals sum A grad m_beta + sum C m_I ^ m,
    checked pointwise at random points (an identity of polynomials)."""
    rng = np.random.default_rng(k)
    xP = rng.uniform(-1, 1, 3)
    hP = 0.7
    X = xP + rng.uniform(-1, 1, (50, 3))
    vecs, grads, crosses, A, C = decompose(k, hP)
    G = eval_grad_mono3(grads, X, xP, hP)                        # (N, ng, 3)
    W = np.stack([mI_cross(c, a, X, xP, hP) for (c, a) in crosses], 1) if crosses else np.zeros((50, 0, 3))
    for r, (c, a) in enumerate(vecs):
        lhs = np.zeros((50, 3))
        lhs[:, c] = eval_mono3([a], X, xP, hP)[:, 0]
        rhs = np.einsum("j,njd->nd", A[r], G) + np.einsum("j,njd->nd", C[r], W)
        np.testing.assert_allclose(rhs, lhs, atol=1e-12)


def test_prop21_coefficients_as_printed():
    """Prop 2.1 for alpha = (1,2,3): h/(|a|+1) on grad m_(2,2,3),
    -alpha_3/(|a|+1) on m_I ^ (0, m_(1,2,2), 0), +alpha_2/(|a|+1) on
    m_I ^ (0, 0, m_(1,1,3)) (the last two rewritten into M^{G,+} only when
    they are x-components, which they are not)."""
    h = 0.37
    vecs, grads, crosses, A, C = decompose(6, h)
    r = vecs.index((0, (1, 2, 3)))
    assert A[r, grads.index((2, 2, 3))] == pytest.approx(h / 7)
    assert np.count_nonzero(A[r]) == 1
    assert C[r, crosses.index((1, (1, 2, 2)))] == pytest.approx(-3 / 7)
    assert C[r, crosses.index((2, (1, 1, 3)))] == pytest.approx(2 / 7)
    assert np.count_nonzero(C[r]) == 2


def test_prop24_identity():
    """Prop 2.4: m_I ^ (m_a,0,0) = -m_I ^ (0,m_b,0) - m_I ^ (0,0,m_g)."""
    rng = np.random.default_rng(3)
    X = rng.uniform(-1, 1, (40, 3))
    xP = np.zeros(3)
    for a in [(1, 0, 0), (2, 1, 0), (1, 1, 2), (3, 0, 1)]:
        b = (a[0] - 1, a[1] + 1, a[2])
        g = (a[0] - 1, a[1], a[2] + 1)
        lhs = mI_cross(0, a, X, xP, 1.0)
        rhs = -mI_cross(1, b, X, xP, 1.0) - mI_cross(2, g, X, xP, 1.0)
        np.testing.assert_allclose(lhs, rhs, atol=1e-14)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
def test_dimensions(k):
    """eq. dimGperp and eq. dimMAndG: dim M^{G,+}_{k-1} = (2k^3+9k^2+7k)/6 and
    dim G_k = dim P_{k+1} - 1 (the corrected form of the dimension count)."""
    assert len(MG_plus(k - 1)) * 6 == 2 * k ** 3 + 9 * k ** 2 + 7 * k
    vecs, grads, crosses, A, C = decompose(k, 1.0)
    assert len(grads) == dim_P3(k + 1) - 1
    assert len(vecs) == len(grads) + len(crosses)   # eq. spaceDec: a direct sum


@pytest.mark.parametrize("k", [1, 2, 3])
def test_cross_set_is_a_basis_of_gperp(k):
    """m_I ^ M^{G,+}_{k-1} is linearly independent and, together with the
    gradients of M_{k+1} minus constants, spans [P_k]^3 (rank test on values)."""
    rng = np.random.default_rng(k + 10)
    X = rng.uniform(-1, 1, (400, 3))
    xP = np.zeros(3)
    vecs, grads, crosses, A, C = decompose(k, 1.0)
    G = eval_grad_mono3(grads, X, xP, 1.0)
    W = np.stack([mI_cross(c, a, X, xP, 1.0) for (c, a) in crosses], 1)
    basis = np.concatenate([G, W], 1).transpose(0, 2, 1).reshape(-1, len(grads) + len(crosses))
    assert np.linalg.matrix_rank(basis) == len(vecs)
    assert np.linalg.matrix_rank(W.transpose(0, 2, 1).reshape(-1, len(crosses))) == len(crosses)


def test_N_set_needs_the_constant():
    """With 0 < |alpha| in eq. NDef, dim M^{G,+}_0 would be 2; the DOF counts of
    Tables 1-3 need 3 cross moments per cell at k = 1."""
    assert len(MG_plus(0)) == 3
    assert sum(1 for a in mono3(0) if a[0] == 0 and sum(a) > 0) + 2 == 2
