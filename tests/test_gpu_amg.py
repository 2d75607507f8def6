"""Parity of the library's smoothed-aggregation AMG (inner solver for S)
with oracle/amg.py on the same seeded inputs: the hierarchy (levels, sizes,
aggregates bit for bit, coarse operators and prolongators to rounding), one
V-cycle, and solves with the AMG inner solver against the oracle's direct
solve.  The oracle builds its hierarchy from its own S, so both sides take
every integer decision from independently computed FP64 values."""

import numpy as np
import pytest

from oracle import E0, amg, assemble, paper_element, solvers
from synth import fields, hex_mesh, prism_mesh
from synth.voronoi import voronoi_mesh

pytestmark = pytest.mark.gpu

CASES = {
    "hex10-E0-lognormal": lambda: (hex_mesh(10), E0, 0, fields.K_lognormal(1000, seed=3, sigma=1.0)),
    "hex12-K1-uniform": lambda: (hex_mesh(12), paper_element(1), 1, np.ones(1728)),
    "cvt400-E0-contrast": lambda: _cvt(400, 6, 2.0),
    "prism4-K1-contrast": lambda: _prism(4),
}


# Relative tolerance of prolongator entries and cycle outputs.  The two
# sides build S independently; on hex meshes its entries agree to rounding,
# on the high-contrast polyhedral meshes small entries of S (tiny faces, low
# K) agree only to ~1e-10 relative (the global-matrix parity bounds entries by
# 1e-12 of the largest), and the ratios a_ij / a_ii in P inherit that.
TOL = {"hex10-E0-lognormal": 1e-12, "hex12-K1-uniform": 1e-12, "cvt400-E0-contrast": 1e-9,
       "prism4-K1-contrast": 1e-9}


def _cvt(n, seed, decades):
    m = voronoi_mesh(n, seed=seed, lloyd=4)
    return m, E0, 0, fields.K_high_contrast(m.n_cells, seed=seed, decades=decades)


def _prism(n):
    m = prism_mesh(n)
    return m, paper_element(1), 1, fields.K_high_contrast(m.n_cells, seed=2, decades=3.0)


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    import torch
    assert torch.cuda.is_available()
    return vemsolve


def _pair(vs, name, **kw):
    mesh, spec, elem, K = CASES[name]()
    prob = fields.sine_problem()
    s = vs.Solver(mesh, element=elem, inner=vs.VEM_INNER_AMG, **kw)
    s.set_coefficient(K)
    s.set_data(prob.f, prob.gD)
    sys_ = assemble(mesh, spec, 1.0 / K, f=prob.f, gD=prob.gD)
    return s, sys_


@pytest.mark.parametrize("name", list(CASES))
def test_hierarchy_matches_oracle(vs, name):
    s, sys_ = _pair(vs, name)
    try:
        s.amg_setup()
        rows, nnz, _ = s.amg_levels()
        H = amg.setup(solvers.schur(sys_))
        assert list(rows) == H.sizes, (list(rows), H.sizes)
        for lvl, ref in enumerate(H.levels):
            A, agg, P = s.amg_level(lvl)
            d = abs(A - ref.A)
            assert d.max() <= 1e-11 * abs(ref.A).max(), (lvl, d.max())
            if ref.P is not None:
                np.testing.assert_array_equal(agg, ref.agg)
                dp = abs(P - ref.P)
                assert dp.max() <= TOL[name] * abs(ref.P).max(), (lvl, dp.max())
    finally:
        s.close()


@pytest.mark.parametrize("name", ["hex10-E0-lognormal", "cvt400-E0-contrast"])
def test_vcycle_matches_oracle(vs, name):
    import torch
    s, sys_ = _pair(vs, name)
    try:
        s.amg_setup()
        H = amg.setup(solvers.schur(sys_))
        n = sys_.n_p
        b = np.random.default_rng(11).standard_normal(n)
        xb = torch.from_numpy(b).cuda()
        x = torch.empty_like(xb)
        s.amg_vcycle_device(xb, x)
        ref = amg.vcycle(H, b)
        err = np.abs(x.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 10 * TOL[name], err
    finally:
        s.close()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("krylov,prec", [(0, 0), (1, 1)], ids=["minres-diag", "fgmres-tri"])
def test_solve_with_amg_matches_direct(vs, name, krylov, prec):
    s, sys_ = _pair(vs, name, krylov=krylov, precond=prec, rtol=1e-12, inner_rtol=1e-13)
    try:
        u, p, st = s.solve()
    finally:
        s.close()
    ud, pd = solvers.solve_direct(sys_)
    assert st["relres"] <= 1e-12
    assert st["amg_levels"] >= 1
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-10 * np.linalg.norm(pd)


def test_amg_cuts_inner_iterations(vs):
    mesh = hex_mesh(24)
    K = fields.K_lognormal(mesh.n_cells, seed=4, sigma=1.5)
    prob = fields.sine_problem()
    its = {}
    for inner in (vs.VEM_INNER_PCG, vs.VEM_INNER_AMG):
        s = vs.Solver(mesh, element=0, krylov=1, precond=1, rtol=1e-10, inner_rtol=1e-10, inner=inner)
        s.set_coefficient(K)
        s.set_data(prob.f, prob.gD)
        _, _, st = s.solve()
        s.close()
        its[inner] = st["inner_iterations"]
        assert st["relres"] <= 1e-10
    assert its[vs.VEM_INNER_AMG] * 4 < its[vs.VEM_INNER_PCG], its


def test_single_level_is_exact(vs):
    """64 cells: S itself is the coarsest level (dense inverse), so the
    AMG-preconditioned CG converges in one iteration per inner solve."""
    mesh = hex_mesh(4)
    prob = fields.sine_problem()
    s = vs.Solver(mesh, element=0, krylov=1, precond=1, rtol=1e-12, inner_rtol=1e-12, inner=vs.VEM_INNER_AMG)
    s.set_coefficient(fields.K_lognormal(64, seed=1))
    s.set_data(prob.f, prob.gD)
    _, _, st = s.solve()
    s.close()
    assert st["amg_levels"] == 1
    assert st["inner_iterations"] <= 2 * st["iterations"] + 2, st


def test_deterministic_hierarchy_and_solve(vs):
    outs = []
    for _ in range(2):
        s, _ = _pair(vs, "cvt400-E0-contrast", krylov=1, precond=1, rtol=1e-11, inner_rtol=1e-11)
        u, p, st = s.solve()
        A1, agg0, P0 = s.amg_level(1)[0], s.amg_level(0)[1], s.amg_level(0)[2]
        s.close()
        outs.append((u, p, A1, agg0, P0))
    a, b = outs
    np.testing.assert_array_equal(a[0], b[0])
    np.testing.assert_array_equal(a[1], b[1])
    assert (a[2] != b[2]).nnz == 0 and (a[4] != b[4]).nnz == 0
    np.testing.assert_array_equal(a[3], b[3])


@pytest.mark.parametrize("name", ["hex10-E0-lognormal", "cvt400-E0-contrast", "prism4-K1-contrast"])
def test_fp32_cycle(vs, name):
    """Mixed option: FP32 V-cycle inside the FP64 CG.  One cycle matches the
    oracle's FP64 cycle to FP32 rounding; the solve still reaches the FP64
    tolerance and the oracle's direct solution."""
    import torch
    s, sys_ = _pair(vs, name, krylov=1, precond=1, rtol=1e-11, inner_rtol=1e-11,
                    precision=vs.VEM_PRECISION_MIXED)
    try:
        s.amg_setup()
        H = amg.setup(solvers.schur(sys_))
        b = np.random.default_rng(12).standard_normal(sys_.n_p)
        xb = torch.from_numpy(b).cuda()
        x = torch.empty_like(xb)
        s.amg_vcycle_device(xb, x)
        ref = amg.vcycle(H, b)
        err = np.abs(x.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 1e-4, err
        u, p, st = s.solve()
    finally:
        s.close()
    ud, pd = solvers.solve_direct(sys_)
    assert st["relres"] <= 1e-11
    assert np.linalg.norm(u - ud) <= 1e-9 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-9 * np.linalg.norm(pd)


def test_unsupported_combinations(vs):
    mesh = hex_mesh(3)
    s = vs.Solver(mesh, element=0, krylov=1, precond=1, inner=vs.VEM_INNER_AMG)
    try:
        with pytest.raises(vs.VemError) as e:
            s.solve_batched(np.ones((2, mesh.n_cells)))
        assert e.value.code == 8
        with pytest.raises(vs.VemError):
            s.amg_levels()
    finally:
        s.close()


@pytest.mark.parametrize("name", ["hex10-E0-lognormal", "cvt400-E0-contrast", "prism4-K1-contrast"])
def test_chebyshev_option_vcycle_matches_oracle(vs, name):
    """inner_smoother = Chebyshev: the same hierarchy with two Chebyshev steps
    of the Jacobi iteration before and after the coarse correction; one cycle
    against the oracle's Chebyshev cycle."""
    import torch
    s, sys_ = _pair(vs, name, inner_smoother=vs.VEM_SMOOTH_CHEBYSHEV)
    try:
        s.amg_setup()
        H = amg.setup(solvers.schur(sys_), smoother="chebyshev")
        assert list(s.amg_levels()[0]) == H.sizes
        b = np.random.default_rng(13).standard_normal(sys_.n_p)
        xb = torch.from_numpy(b).cuda()
        x = torch.empty_like(xb)
        s.amg_vcycle_device(xb, x)
        ref = amg.vcycle(H, b)
        err = np.abs(x.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 10 * TOL[name], err
    finally:
        s.close()


@pytest.mark.parametrize("name", ["hex10-E0-lognormal", "cvt400-E0-contrast", "hex12-K1-uniform"])
@pytest.mark.parametrize("krylov,prec", [(0, 0), (1, 1)], ids=["minres-diag", "fgmres-tri"])
def test_chebyshev_option_solve_matches_direct(vs, name, krylov, prec):
    s, sys_ = _pair(vs, name, krylov=krylov, precond=prec, rtol=1e-12, inner_rtol=1e-13,
                    inner_smoother=vs.VEM_SMOOTH_CHEBYSHEV)
    try:
        u, p, st = s.solve()
    finally:
        s.close()
    ud, pd = solvers.solve_direct(sys_)
    assert st["relres"] <= 1e-12
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-10 * np.linalg.norm(pd)


def test_chebyshev_option_cuts_inner_iterations(vs):
    """The oracle's AMG-PCG needs about 0.6 of the Jacobi-smoothed iterations
    with the Chebyshev smoother on these operators; the library likewise."""
    mesh = hex_mesh(24)
    K = fields.K_lognormal(mesh.n_cells, seed=4, sigma=1.5)
    prob = fields.sine_problem()
    its = {}
    for sm in (vs.VEM_SMOOTH_JACOBI, vs.VEM_SMOOTH_CHEBYSHEV):
        s = vs.Solver(mesh, element=0, krylov=1, precond=1, rtol=1e-10, inner_rtol=1e-10, inner=vs.VEM_INNER_AMG,
                      inner_smoother=sm)
        s.set_coefficient(K)
        s.set_data(prob.f, prob.gD)
        _, _, st = s.solve()
        s.close()
        its[sm] = st["inner_iterations"]
        assert st["relres"] <= 1e-10
    assert its[vs.VEM_SMOOTH_CHEBYSHEV] < 0.8 * its[vs.VEM_SMOOTH_JACOBI], its
