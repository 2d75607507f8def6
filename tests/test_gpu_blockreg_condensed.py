"""Parity of Block-Reg's condensed cycle (reg_cycle = VEM_REG_CONDENSED, the
paper's k = 1 element; Sec. 5, eq. block_diag with the flux block A_reg =
A + B^T B / gamma) with oracle/block_amg.CondensedCycle: the face system
S_f = A_ff - A_fi A_ii^-1 A_if, its point-block hierarchy (3 x 3 face
blocks, the face DOFs of the constant fields as near-null space, Chebyshev
smoothing: level sizes, block aggregates bit for bit, operators and
prolongators to rounding), the whole condensed cycle on a vector of A_reg's
size, Block-Reg solves against the oracle's direct solve and outer iteration
counts against the oracle's Krylov solve with the same cycle."""

import os

import numpy as np
import pytest

from oracle import assemble, block_amg, paper_element, solvers
from synth import fields, hex_mesh, octa_mesh
from synth.voronoi import voronoi_mesh

pytestmark = pytest.mark.gpu

K1 = paper_element(1)
PROCS = max(1, min(16, os.cpu_count() or 1))


def _flux(m):
    m.face_bc = np.where(m.face_bc != 0, 2, 0).astype(np.int8)
    return m


CASES = {
    "hex5-lognormal": lambda: (hex_mesh(5), fields.K_lognormal(125, seed=3, sigma=1.0), False),
    "hex5-flux": lambda: (_flux(hex_mesh(5)), np.ones(125), True),
    "hex8-flux": lambda: (_flux(hex_mesh(8)), np.ones(512), True),
    "octa2-flux": lambda: (octa_mesh(2, bc=2), np.ones(72), True),
    "cvt125-flux": lambda: _cvt(125),
}
# Tolerances relative to the largest entry: A_reg's local flux matrices of
# the two sides agree to rounding on structured cells and to ~1e-10 on
# Voronoi cells with tiny faces.
TOL = {"hex5-lognormal": 1e-11, "hex5-flux": 1e-11, "hex8-flux": 1e-11, "octa2-flux": 1e-11, "cvt125-flux": 1e-8}


def _cvt(n):
    m = _flux(voronoi_mesh(n, seed=7, lloyd=10))
    return m, np.ones(m.n_cells), True


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    import torch
    assert torch.cuda.is_available()
    return vemsolve


def _pair(vs, name, **kw):
    mesh, K, flux = CASES[name]()
    prob = fields.paper_polynomial_problem()
    s = vs.Solver(mesh, element=1, precond=vs.VEM_PREC_BLOCK_REG, reg_cycle=vs.VEM_REG_CONDENSED, **kw)
    s.set_coefficient(K)
    fl = prob.u if flux else None
    s.set_data(prob.f, prob.gD, flux=fl)
    sys_ = assemble(mesh, K1, 1.0 / K, f=prob.f, gD=prob.gD, flux=fl, keep_local=True, processes=PROCS)
    return s, sys_


def _cycle(sys_):
    return block_amg.CondensedCycle(sys_, solvers.regularized(sys_, solvers.mesh_size(sys_) ** 2))


@pytest.mark.parametrize("name", list(CASES))
def test_face_system_and_hierarchy(vs, name):
    s, sys_ = _pair(vs, name)
    try:
        s.amg_setup(vs.VEM_AMG_REG)
        cc = _cycle(sys_)
        rows, _, _ = s.amg_levels(vs.VEM_AMG_REG)
        assert rows[0] == cc.nf
        assert list(rows) == cc.H.sizes, (list(rows), cc.H.sizes)
        for lvl, ref in enumerate(cc.H.levels):
            A, agg, P = s.amg_level(lvl, vs.VEM_AMG_REG)
            assert abs(A - ref.A).max() <= TOL[name] * abs(ref.A).max(), lvl
            if ref.P is not None:
                nb = ref.A.shape[0] // ref.bs
                np.testing.assert_array_equal(agg[:nb], ref.agg)
                assert abs(P - ref.P).max() <= 10 * TOL[name] * abs(ref.P).max(), lvl
    finally:
        s.close()


@pytest.mark.parametrize("name", ["hex5-lognormal", "hex8-flux", "cvt125-flux"])
def test_condensed_cycle_matches_oracle(vs, name):
    """The whole cycle: interior elimination, the face V-cycle, recovery."""
    import torch
    s, sys_ = _pair(vs, name)
    try:
        s.amg_setup(vs.VEM_AMG_REG)
        cc = _cycle(sys_)
        r = np.random.default_rng(23).standard_normal(sys_.n_u)
        rb = torch.from_numpy(r).cuda()
        x = torch.empty_like(rb)
        s.amg_vcycle_device(rb, x, vs.VEM_AMG_REG)
        ref = cc(r)
        err = np.abs(x.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err <= 100 * TOL[name], err
    finally:
        s.close()


@pytest.mark.parametrize("name", ["hex5-lognormal", "hex5-flux", "octa2-flux", "cvt125-flux"])
@pytest.mark.parametrize("krylov", [0, 1], ids=["minres", "fgmres"])
def test_condensed_solve_matches_direct(vs, name, krylov):
    s, sys_ = _pair(vs, name, krylov=krylov, rtol=1e-11, maxit=4000)
    try:
        u, p, st = s.solve()
    finally:
        s.close()
    ud, pd = solvers.solve_direct(sys_)
    assert st["relres"] <= 1e-11
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-8 * np.linalg.norm(pd)


@pytest.mark.parametrize("name", ["hex5-flux", "hex8-flux", "cvt125-flux"])
def test_condensed_iterations_match_oracle(vs, name):
    """FGMRES(30) with the same cycle: the outer counts agree to a few
    iterations (rounding differs), and they are far below the scalar cycle's."""
    s, sys_ = _pair(vs, name, krylov=1, restart=30, rtol=1e-8, maxit=4000)
    try:
        _, _, st = s.solve()
        s.set_options(reg_cycle=vs.VEM_REG_SCALAR_AMG)
        _, _, st_scalar = s.solve()
    finally:
        s.close()
    _, _, res = solvers.solve_krylov(sys_, "fgmres", "reg", rtol=1e-8, restart=30, maxit=4000,
                                     reg_smoother="condensed-block")
    assert res.converged
    assert abs(st["iterations"] - res.iters) <= max(3, 0.1 * res.iters), (st["iterations"], res.iters)
    assert st["iterations"] < st_scalar["iterations"], (st["iterations"], st_scalar["iterations"])


def test_condensed_unsupported(vs):
    mesh = hex_mesh(3)
    prob = fields.sine_problem()
    for kw in (dict(element=0), dict(element=2), dict(element=1, precision=1)):
        s = vs.Solver(mesh, krylov=1, precond=vs.VEM_PREC_BLOCK_REG, reg_cycle=vs.VEM_REG_CONDENSED, **kw)
        try:
            s.set_data(prob.f, prob.gD)
            with pytest.raises(vs.VemError) as e:
                s.solve()
            assert e.value.code == 8
        finally:
            s.close()
