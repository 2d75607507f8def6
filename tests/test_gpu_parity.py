"""Parity of the CUDA path (through the C-ABI) with the CPU oracle on the same
seeded inputs: geometry, local matrices (Sec. 4.3), the assembled saddle
system and Schur approximation (Sec. 5), and solutions (MINRES / FGMRES with
the block preconditioners) against the oracle's direct solve."""

import numpy as np
import pytest

from oracle import E0, assemble, paper_element, solvers
from oracle.assemble import mesh_cells
from oracle.element import local_system
from synth import affine, fields, hex_mesh, octa_mesh, prism_mesh, tet_mesh
from synth.voronoi import voronoi_mesh

pytestmark = pytest.mark.gpu

A_SHEAR = np.array([[1.0, 0.3, 0.1], [0.0, 0.8, -0.2], [0.1, 0.0, 1.2]])
MESHES = {
    "hex3": lambda: hex_mesh(3),
    "tet2": lambda: tet_mesh(2),
    "prism2": lambda: prism_mesh(2),
    "sheared": lambda: affine(hex_mesh(2), A_SHEAR, (0.1, 0.0, -0.3)),
    "octa2": lambda: octa_mesh(2),
    "cvt": lambda: voronoi_mesh(40, seed=3, lloyd=5),
}
ELEMENTS = {"E0": (E0, 0), "K1": (paper_element(1), 1)}


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    import torch
    assert torch.cuda.is_available()
    return vemsolve


def _solver(vs, mesh, elem, **kw):
    return vs.Solver(mesh, element=elem, **kw)


@pytest.mark.parametrize("mname", list(MESHES))
def test_geometry(vs, mname):
    mesh = MESHES[mname]()
    s = _solver(vs, mesh, 0)
    g = s.geometry()
    cells = mesh_cells(mesh)
    np.testing.assert_allclose(g["cell_volume"], [c.volume for c in cells], rtol=1e-13)
    np.testing.assert_allclose(g["cell_centroid"], [c.centroid for c in cells], atol=1e-14)
    np.testing.assert_allclose(g["cell_diam"], [c.diameter for c in cells], rtol=1e-14)
    from oracle.polyhedron import face_geometry
    F = [face_geometry(mesh, f) for f in range(mesh.n_faces)]
    np.testing.assert_allclose(g["face_area"], [x.area for x in F], rtol=1e-13)
    np.testing.assert_allclose(g["face_centroid"], [x.centroid for x in F], atol=1e-14)
    np.testing.assert_allclose(g["face_normal"], [x.normal for x in F], atol=1e-14)
    s.close()


@pytest.mark.parametrize("mname", list(MESHES))
@pytest.mark.parametrize("ename", list(ELEMENTS))
def test_local_matrices(vs, mname, ename):
    spec, elem = ELEMENTS[ename]
    mesh = MESHES[mname]()
    K = fields.K_lognormal(mesh.n_cells, seed=3, sigma=1.0)
    s = _solver(vs, mesh, elem)
    s.set_coefficient(K)
    s.assemble()
    loc = s.local_matrices()
    cells = mesh_cells(mesh)
    for c, cell in enumerate(cells):
        ref = local_system(cell, spec, 1.0 / K[c])
        M, B = loc[c]
        scale = np.abs(ref["M"]).max()
        np.testing.assert_allclose(M, ref["M"], rtol=0, atol=1e-12 * scale, err_msg=f"cell {c}")
        np.testing.assert_allclose(B, ref["B"][0], rtol=0, atol=1e-12 * np.abs(ref["B"]).max())
    s.close()


def _oracle_system(mesh, spec, K, prob):
    return assemble(mesh, spec, 1.0 / K, f=prob.f, gD=prob.gD)


@pytest.mark.parametrize("mname", ["hex3", "prism2", "sheared", "cvt"])
@pytest.mark.parametrize("ename", list(ELEMENTS))
def test_global_system_and_schur(vs, mname, ename):
    spec, elem = ELEMENTS[ename]
    mesh = MESHES[mname]()
    K = fields.K_lognormal(mesh.n_cells, seed=5, sigma=1.0)
    prob = fields.quadratic_problem()
    s = _solver(vs, mesh, elem)
    s.set_coefficient(K)
    s.set_data(prob.f, prob.gD)
    A, rhs = s.system()
    sys = _oracle_system(mesh, spec, K, prob)
    Ar = sys.saddle()
    d = (A - Ar).toarray()
    assert np.abs(d).max() <= 1e-12 * np.abs(Ar).max()
    np.testing.assert_allclose(rhs, sys.rhs(), rtol=0, atol=1e-12 * np.abs(sys.rhs()).max())
    S, dM = s.schur()
    Sr = solvers.schur(sys)
    assert np.abs((S - Sr).toarray()).max() <= 1e-12 * np.abs(Sr).max()
    # exact integrals by two different schemes: rounding-level differences only
    np.testing.assert_allclose(dM, sys.M.diagonal(), rtol=1e-11)
    s.close()


SOLVES = [("minres", 0, 0), ("fgmres", 1, 0), ("fgmres", 1, 1)]


@pytest.mark.parametrize("mname", list(MESHES))
@pytest.mark.parametrize("ename", list(ELEMENTS))
@pytest.mark.parametrize("method,krylov,prec", SOLVES, ids=["minres-diag", "fgmres-diag", "fgmres-tri"])
def test_solve_matches_oracle_direct(vs, mname, ename, method, krylov, prec):
    """FP64 GPU solution vs the oracle's direct solve: <= 1e-10 relative at a
    true relative residual <= 1e-12."""
    spec, elem = ELEMENTS[ename]
    mesh = MESHES[mname]()
    K = fields.K_lognormal(mesh.n_cells, seed=7, sigma=1.0)
    prob = fields.sine_problem()
    s = _solver(vs, mesh, elem, krylov=krylov, precond=prec, rtol=1e-12, inner_rtol=1e-13)
    s.set_coefficient(K)
    s.set_data(prob.f, prob.gD)
    u, p, st = s.solve()
    sys = _oracle_system(mesh, spec, K, prob)
    ud, pd = solvers.solve_direct(sys)
    assert st["relres"] <= 1e-12
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-10 * np.linalg.norm(pd)
    s.close()


@pytest.mark.parametrize("n_side", [12, 17], ids=["one-block-pcg", "multi-launch-pcg"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_inner_pcg_both_forms(vs, n_side, precision):
    """The inner Jacobi-PCG runs in one thread block for S of up to 4,096
    rows and 16,384 stored entries (12^3 cells: 1,728 rows, 7-point rows)
    and as launches of its multi-block kernels above (17^3: 4,913 rows):
    both forms reach the oracle's direct solution with a general right-hand
    side (FP64: 1e-10; mixed: FP32 inner solve, FP64 refinement), in FGMRES
    with the block-triangular preconditioner."""
    mesh = hex_mesh(n_side)
    K = fields.K_lognormal(mesh.n_cells, seed=9, sigma=1.0)
    f = np.random.default_rng(3).standard_normal(mesh.n_cells)
    s = _solver(vs, mesh, 0, krylov=1, precond=1, rtol=1e-12, inner_rtol=1e-6, maxit=500,
                precision=precision)
    try:
        s.set_coefficient(K)
        s.set_source(f, None)
        u, p, st = s.solve()
    finally:
        s.close()
    sys = assemble(mesh, E0, 1.0 / K)
    cells = mesh_cells(mesh)
    sys.F[:] = [c.volume * f[i] for i, c in enumerate(cells)]
    ud, pd = solvers.solve_direct(sys)
    assert st["relres"] <= 1e-12
    assert st["inner_iterations"] >= st["iterations"]
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-10 * np.linalg.norm(pd)


def test_random_rhs_krylov(vs):
    """A right-hand side with no special structure (the manufactured sine data
    is an eigenvector on uniform cubes): FGMRES + block-triangular needs tens of
    iterations and still matches the direct solve."""
    mesh = hex_mesh(6)
    K = fields.K_lognormal(mesh.n_cells, seed=8, sigma=1.0)
    rng = np.random.default_rng(1)
    f = rng.standard_normal(mesh.n_cells)
    s = _solver(vs, mesh, 1, krylov=1, precond=1, rtol=1e-12, inner_rtol=1e-10)
    s.set_coefficient(K)
    s.set_source(f, None)
    u, p, st = s.solve()
    sys = assemble(mesh, paper_element(1), 1.0 / K)
    cells = mesh_cells(mesh)
    sys.F[:] = [c.volume * f[i] for i, c in enumerate(cells)]
    ud, pd = solvers.solve_direct(sys)
    assert st["iterations"] > 10
    assert np.linalg.norm(u - ud) <= 1e-10 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-10 * np.linalg.norm(pd)


def test_one_cell_mesh(vs):
    mesh = hex_mesh(1)
    prob = fields.linear_problem()
    for elem, spec in ((0, E0), (1, paper_element(1))):
        s = _solver(vs, mesh, elem, krylov=1, precond=1)
        s.set_data(prob.f, prob.gD)
        u, p, st = s.solve()
        sys = _oracle_system(mesh, spec, np.ones(1), prob)
        ud, pd = solvers.solve_direct(sys)
        np.testing.assert_allclose(u, ud, atol=1e-12)
        np.testing.assert_allclose(p, pd, atol=1e-12)


def test_bad_inputs(vs):
    mesh = hex_mesh(2)
    s = _solver(vs, mesh, 0)
    with pytest.raises(vs.VemError) as e:
        s.set_coefficient(np.r_[np.ones(7), -1.0])
    assert e.value.code == 1
    with pytest.raises(vs.VemError) as e:
        s.set_source(np.r_[np.ones(7), np.nan], None)
    assert e.value.code == 5
    with pytest.raises(vs.VemError) as e:
        vs.Solver(mesh, element=7)
    assert e.value.code == 1
    # MINRES with the non-symmetric preconditioner is refused
    with pytest.raises(vs.VemError):
        vs.Solver(mesh, krylov=0, precond=1)


def test_not_converged_status(vs):
    mesh = hex_mesh(4)
    rng = np.random.default_rng(3)
    s = _solver(vs, mesh, 1, krylov=1, precond=0, maxit=2, rtol=1e-14)
    s.set_source(rng.standard_normal(mesh.n_cells), None)
    with pytest.raises(vs.VemError) as e:
        s.solve()
    assert e.value.code == 3
    u, p, st = s.solve(allow_not_converged=True)
    assert st["iterations"] == 2 and st["relres"] > 1e-14


def test_degenerate_face(vs):
    mesh = hex_mesh(2)
    # collapse one boundary face onto a segment: its area vanishes
    xyz = mesh.xyz.copy()
    f = int(np.nonzero(mesh.face_bc)[0][0])
    vid = mesh.face_vertices(f)
    xyz[vid[2]] = xyz[vid[1]]
    xyz[vid[3]] = xyz[vid[0]]
    bad = type(mesh)(xyz, mesh.face_vtx_ptr, mesh.face_vtx, mesh.cell_face_ptr, mesh.cell_face, mesh.face_bc)
    with pytest.raises(vs.VemError) as e:
        vs.Solver(bad)
    assert e.value.code == 2


def test_deterministic(vs):
    mesh = prism_mesh(3)
    rng = np.random.default_rng(4)
    f = rng.standard_normal(mesh.n_cells)
    out = []
    for _ in range(2):
        s = _solver(vs, mesh, 1, krylov=1, precond=1, inner_rtol=1e-8)
        s.set_source(f, None)
        out.append(s.solve())
        s.close()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("mname", ["hex3", "tet2", "sheared", "cvt"])
@pytest.mark.parametrize("ename", list(ELEMENTS))
def test_mixed_precision_refinement(vs, mname, ename):
    """FP32 preconditioner / inner Schur solve with the FP64 outer FGMRES: the
    true FP64 residual still reaches 1e-10 and the solution matches the FP64
    oracle within 1e-8 (relative), on a high-contrast K = 10^U, U in [-4, 4]."""
    spec, elem = ELEMENTS[ename]
    mesh = MESHES[mname]()
    K = fields.K_high_contrast(mesh.n_cells, seed=1)
    prob = fields.sine_problem()
    s = _solver(vs, mesh, elem, krylov=1, precond=1, precision=vs.VEM_PRECISION_MIXED, rtol=1e-10,
                inner_rtol=1e-5, maxit=500)
    s.set_coefficient(K)
    s.set_data(prob.f, prob.gD)
    u, p, st = s.solve()
    sys = _oracle_system(mesh, spec, K, prob)
    ud, pd = solvers.solve_direct(sys)
    assert st["relres"] <= 1e-10
    assert np.linalg.norm(u - ud) <= 1e-8 * np.linalg.norm(ud)
    assert np.linalg.norm(p - pd) <= 1e-8 * np.linalg.norm(pd)
    s.close()


def test_mixed_precision_needs_fgmres(vs):
    with pytest.raises(vs.VemError) as e:
        vs.Solver(hex_mesh(2), krylov=0, precond=0, precision=vs.VEM_PRECISION_MIXED)
    assert e.value.code == 1


@pytest.mark.parametrize("mname,expect_few", [("hex3", True), ("sheared", True), ("cvt", False)])
@pytest.mark.parametrize("ename", list(ELEMENTS))
def test_reuse_of_congruent_cells(vs, mname, expect_few, ename):
    """Cells that are translates of one another share one evaluation of their
    geometry-only local matrices: same solution (to rounding) with reuse on
    and off, and the class count is tiny on structured meshes and equals the
    cell count on a Voronoi mesh."""
    spec, elem = ELEMENTS[ename]
    mesh = MESHES[mname]()
    K = fields.K_lognormal(mesh.n_cells, seed=9, sigma=1.0)
    prob = fields.sine_problem()
    out = {}
    for reuse in (1, 0):
        s = _solver(vs, mesh, elem, krylov=1, precond=1, rtol=1e-12, inner_rtol=1e-13, reuse=reuse)
        s.set_coefficient(K)
        s.set_data(prob.f, prob.gD)
        out[reuse] = s.solve()
        s.close()
    (u1, p1, st1), (u0, p0, st0) = out[1], out[0]
    assert st0["n_classes"] == mesh.n_cells
    if expect_few:
        assert st1["n_classes"] <= 3
    else:
        assert st1["n_classes"] == mesh.n_cells
    assert np.linalg.norm(u1 - u0) <= 1e-11 * np.linalg.norm(u0)
    assert np.linalg.norm(p1 - p0) <= 1e-11 * np.linalg.norm(p0)


def test_bad_mesh_inputs(vs):
    """The mesh is checked on the device before any kernel follows its
    indices: out-of-range vertex and face ids, short faces and cells, face
    flags and coordinates are refused with a status, and the device stays
    usable (a valid mesh solves afterwards)."""
    mesh = hex_mesh(2)

    def variant(**kw):
        a = dict(xyz=mesh.xyz.copy(), fvp=mesh.face_vtx_ptr.copy(), fv=mesh.face_vtx.copy(),
                 cfp=mesh.cell_face_ptr.copy(), cf=mesh.cell_face.copy(), bc=mesh.face_bc.copy())
        a.update(kw)
        return type(mesh)(a["xyz"], a["fvp"], a["fv"], a["cfp"], a["cf"], a["bc"])

    fv = mesh.face_vtx.copy()
    fv[5] = mesh.n_vertices + 3
    cf = mesh.cell_face.copy()
    cf[2] = -1
    bc = mesh.face_bc.copy()
    bc[0] = 7
    xyz = mesh.xyz.copy()
    xyz[4, 1] = np.nan
    # first face with two vertices: move one vertex id to the next face
    fvp = mesh.face_vtx_ptr.copy()
    fvp[1] = 2
    cfp = mesh.cell_face_ptr.copy()
    cfp[1] = 3
    cases = [(variant(fv=fv), 1), (variant(cf=cf), 1), (variant(bc=bc), 1), (variant(xyz=xyz), 5),
             (variant(fvp=fvp), 1), (variant(cfp=cfp), 1)]
    for bad, code in cases:
        with pytest.raises(vs.VemError) as e:
            vs.Solver(bad)
        assert e.value.code == code, (e.value, code)
    prob = fields.sine_problem()
    s = _solver(vs, mesh, 0, krylov=1, precond=1, rtol=1e-10, inner_rtol=1e-12)
    try:
        s.set_data(prob.f, prob.gD)
        _, _, st = s.solve()
    finally:
        s.close()
    assert st["relres"] <= 1e-10


def test_memory_pool_reuse_and_release(vs):
    """Handles created after others were destroyed reuse the pool's memory
    and give the same solution bit for bit; releasing the pool's unused
    memory leaves live handles working."""
    mesh = hex_mesh(4)
    prob = fields.sine_problem()
    outs = []
    for _ in range(2):
        s = _solver(vs, mesh, 1, krylov=1, precond=1, rtol=1e-10, inner_rtol=1e-12)
        s.set_data(prob.f, prob.gD)
        outs.append(s.solve()[:2])
        s.close()
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
    np.testing.assert_array_equal(outs[0][1], outs[1][1])
    s = _solver(vs, mesh, 1, krylov=1, precond=1, rtol=1e-10, inner_rtol=1e-12)
    try:
        s.set_data(prob.f, prob.gD)
        vs.release_memory()
        u, p, st = s.solve()
    finally:
        s.close()
    vs.release_memory()
    np.testing.assert_array_equal(u, outs[0][0])
