"""Pins for oracle/amg.py (the smoothed-aggregation AMG for S).

* splitmix64 against the published first outputs of the generator seeded 0;
* the greedy distance-2 independent set against a separately written
  parallel-rounds computation (the form the library runs), plus
  independence and maximality;
* aggregates: a partition of the non-isolated nodes, each node within
  strong distance 2 of its root;
* the two-level correction E = I - P A_c^-1 P^T A is an A-orthogonal
  projector (catches a transposed or mis-scaled P);
* the V-cycle is symmetric positive definite (so it preconditions CG);
* AMG-PCG reaches the direct solution; its iteration count stays bounded
  far below Jacobi-PCG's and grows far more slowly under refinement.
"""

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import E0, amg, assemble, solvers
from synth import fields, hex_mesh
from synth.voronoi import voronoi_mesh


def _lap7(n, nu):
    """S of the lowest-order element on n^3 unit cubes (face weight
    (4a/3)/(nu_P + nu_Q), Dirichlet faces (4a/3)/nu_P); the oracle's own
    assembly is pinned to this form in test_schur_on_uniform_cubes."""
    a = 1.0 / n
    N = n ** 3
    idx = np.arange(N).reshape(n, n, n)
    rows, cols, vals = [], [], []
    diag = np.zeros(N)
    for d in range(3):
        lo = np.take(idx, np.arange(n - 1), axis=d).ravel()
        hi = np.take(idx, np.arange(1, n), axis=d).ravel()
        w = (4 * a / 3) / (nu[lo] + nu[hi])
        rows += [lo, hi]
        cols += [hi, lo]
        vals += [-w, -w]
        np.add.at(diag, lo, w)
        np.add.at(diag, hi, w)
        for b in (np.take(idx, [0], axis=d).ravel(), np.take(idx, [n - 1], axis=d).ravel()):
            np.add.at(diag, b, (4 * a / 3) / nu[b])
    rows.append(np.arange(N))
    cols.append(np.arange(N))
    vals.append(diag)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(N, N))


def test_splitmix64_published_outputs():
    # SplitMix64 seeded with 0: the first three outputs
    g = 0x9E3779B97F4A7C15
    m = (1 << 64) - 1
    assert amg.splitmix64(0) == 0xE220A8397B1DCDAF
    assert amg.splitmix64(g) == 0x6E789E6AA1B965F4
    assert amg.splitmix64((2 * g) & m) == 0x06C45D188009454F


def _rounds_mis2(n, ptr, idx):
    """Parallel rounds: a node joins when its (state, key) is the largest in
    its closed distance-2 ball; a node whose ball holds a member leaves."""
    IN, UND, OUT = 2, 1, 0
    key = np.array([amg.node_key(i) for i in range(n)], dtype=object)
    state = np.full(n, UND)
    nb = [np.concatenate([[i], idx[ptr[i]:ptr[i + 1]]]).astype(int) for i in range(n)]
    for _ in range(10 * n + 10):
        if not (state == UND).any():
            break
        tup = [(state[i], key[i]) for i in range(n)]
        t1 = [max(tup[j] for j in nb[i]) for i in range(n)]
        t2 = [max(t1[j] for j in nb[i]) for i in range(n)]
        new = state.copy()
        for i in range(n):
            if state[i] != UND:
                continue
            if t2[i] == tup[i]:
                new[i] = IN
            elif t2[i][0] == IN:
                new[i] = OUT
        state = new
    assert not (state == UND).any()
    return state == IN


def _graph(A, theta):
    return amg.strength(A, theta)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mis2_greedy_equals_rounds(seed):
    n = 60
    # random symmetric sparse graph with some isolated nodes
    M = sp.random(n, n, density=0.05, random_state=seed)
    M = ((M + M.T) > 0).astype(float)
    M.setdiag(0)
    M.eliminate_zeros()
    A = (sp.diags(np.full(n, 10.0)) - M).tocsr()
    ptr, idx = _graph(A, 0.01)
    g = amg.mis2(n, ptr, idx)
    r = _rounds_mis2(n, ptr, idx)
    np.testing.assert_array_equal(g, r)
    # independence at distance 2 and maximality
    ball = [set([i]) | set(idx[ptr[i]:ptr[i + 1]].tolist()) for i in range(n)]
    ball2 = [set().union(*[ball[j] for j in ball[i]]) for i in range(n)]
    roots = np.nonzero(g)[0]
    for a in roots:
        assert not any(b in ball2[a] for b in roots if b != a)
    for i in range(n):
        assert any(b in ball2[i] for b in roots)


def test_aggregates_partition_and_reach():
    m = voronoi_mesh(300, seed=4, lloyd=3)
    sys_ = assemble(m, E0, fields.K_high_contrast(m.n_cells, seed=2, decades=2.0))
    S = solvers.schur(sys_)
    ptr, idx = amg.strength(S, 0.08)
    agg, nc = amg.aggregate(S.shape[0], ptr, idx)
    iso = np.diff(ptr) == 0
    assert (agg[iso] == -1).all() and (agg[~iso] >= 0).all()
    assert set(agg[~iso].tolist()) == set(range(nc))
    root = amg.mis2(S.shape[0], ptr, idx) & ~iso
    nb = [set(idx[ptr[i]:ptr[i + 1]].tolist()) for i in range(S.shape[0])]
    for i in np.nonzero(~iso)[0]:
        members = np.nonzero(agg == agg[i])[0]
        r = [x for x in members if root[x]]
        if not r:             # a pass-3 singleton
            assert members.size == 1
            continue
        r = r[0]
        assert i == r or r in nb[i] or any(r in nb[j] for j in nb[i])


@pytest.fixture(scope="module")
def lognormal_S():
    n = 12
    nu = 1.0 / fields.K_lognormal(n ** 3, seed=3, sigma=1.0)
    return _lap7(n, nu)


def test_two_level_projector(lognormal_S):
    S = lognormal_S
    H = amg.setup(S, coarse_max=8)
    P = H.levels[0].P.toarray()
    A = S.toarray()
    Ac = H.levels[1].A.toarray()
    E = np.eye(A.shape[0]) - P @ np.linalg.solve(Ac, P.T @ A)
    np.testing.assert_allclose(E @ E, E, atol=1e-9)
    AE = A @ E
    np.testing.assert_allclose(AE, AE.T, atol=1e-9 * np.abs(A).max())
    assert np.linalg.eigvalsh(Ac).min() > 0


def test_vcycle_spd(lognormal_S):
    S = lognormal_S
    H = amg.setup(S)
    n = S.shape[0]
    rng = np.random.default_rng(1)
    U = rng.standard_normal((n, 4))
    V = rng.standard_normal((n, 4))
    MU = np.column_stack([amg.vcycle(H, u) for u in U.T])
    MV = np.column_stack([amg.vcycle(H, v) for v in V.T])
    np.testing.assert_allclose(V.T @ MU, (U.T @ MV).T, rtol=1e-10, atol=1e-10 * np.abs(V.T @ MU).max())
    assert (np.einsum("ij,ij->j", U, MU) > 0).all()


def test_amg_pcg_direct_and_optimality():
    its_amg, its_jac = [], []
    for n in (8, 16, 24):
        nu = 1.0 / fields.K_lognormal(n ** 3, seed=5, sigma=1.0)
        S = _lap7(n, nu)
        b = np.random.default_rng(n).standard_normal(n ** 3)
        H = amg.setup(S)
        r = amg.amg_pcg(S, b, H, rtol=1e-10)
        assert r.converged
        xd = spla.spsolve(S.tocsc(), b)
        assert np.linalg.norm(r.x - xd) <= 1e-8 * np.linalg.norm(xd)
        its_amg.append(r.iters)
        its_jac.append(solvers.pcg(S, b, rtol=1e-10).iters)
    # Jacobi-PCG grows like 1/h; the AMG's count grows far more slowly
    assert its_jac[-1] >= 2 * its_jac[0], its_jac
    assert its_amg[-1] / its_amg[0] <= 0.6 * its_jac[-1] / its_jac[0], (its_amg, its_jac)
    assert its_amg[-1] * 4 < its_jac[-1], (its_amg, its_jac)


def test_schur_of_assembled_system():
    """The AMG on S of the assembled lowest-order system (hex mesh with the
    library's own face order) reaches the direct solution."""
    m = hex_mesh(6)
    sys_ = assemble(m, E0, 1.0 / fields.K_lognormal(m.n_cells, seed=8, sigma=1.5))
    S = solvers.schur(sys_)
    H = amg.setup(S, coarse_max=16)
    assert len(H.levels) >= 2
    b = np.random.default_rng(0).standard_normal(S.shape[0])
    r = amg.amg_pcg(S, b, H, rtol=1e-12)
    assert r.converged and r.relres <= 1e-11
