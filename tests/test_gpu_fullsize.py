"""Full-size parity: the 128^3 paper-k=1 workload (2,097,152 cells,
27,410,432 unknowns) in the launch configuration the benchmark times:
FGMRES(30), block upper-triangular preconditioner, inner AMG-PCG 1e-8,
rtol 1e-8, device-resident inputs and outputs.

The oracle cannot assemble 27 M unknowns, so it builds sampled rows of
[M B^T; B 0] and [g; F] from the local systems (Sec. 4.3) of the cells that
touch them, and the test checks, on those rows:
  1. y = A x for a seeded random x (vem_apply_device) against the oracle's
     rows (the assembled matrix at full size);
  2. the residual of the returned solution (the solve at full size);
and, for all cells, the pressure error against the exact solution, bounded
by the O(h) rate pinned for the oracle (the error of the oracle's own 8^3
solution scaled by 8/128, with a factor 2 of margin)."""

import numpy as np
import pytest

from oracle import paper_element, solvers
from oracle.assemble import assemble, cell_dofmap
from oracle.element import local_system
from oracle.polyhedron import cell_geometry
from synth import fields, hex_mesh

pytestmark = pytest.mark.gpu

N = 128


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    import torch
    assert torch.cuda.is_available()
    return vemsolve


def _oracle_rows(mesh, spec, K, prob, flux_rows, cells_p):
    """Rows {col: val} and rhs entries of the saddle system for the global
    flux DOFs ``flux_rows`` and the pressure rows of ``cells_p``."""
    n_u = spec.nfd * mesh.n_faces + spec.nid * mesh.n_cells
    cf = np.asarray(mesh.cell_face)
    cfp = np.asarray(mesh.cell_face_ptr)
    owner = np.repeat(np.arange(mesh.n_cells), np.diff(cfp))
    order = np.argsort(cf, kind="stable")
    first = np.searchsorted(cf[order], np.arange(mesh.n_faces + 1))

    def cells_of_dof(i):
        if i < spec.nfd * mesh.n_faces:
            f = i // spec.nfd
            return owner[order[first[f]:first[f + 1]]]
        return [(i - spec.nfd * mesh.n_faces) // spec.nid]

    need = set(cells_p.tolist())
    for i in flux_rows:
        need.update(int(c) for c in cells_of_dof(int(i)))
    loc = {}
    for c in sorted(need):
        cell = cell_geometry(mesh, c)
        loc[c] = (local_system(cell, spec, 1.0 / K[c], f=prob.f, gD=prob.gD), cell_dofmap(mesh, c, spec))
    rows, rhs = [], []
    for i in flux_rows:
        row, b = {}, 0.0
        for c in cells_of_dof(int(i)):
            L, dm = loc[int(c)]
            li = int(np.nonzero(dm == i)[0][0])
            for j, v in zip(dm, L["M"][li]):
                row[int(j)] = row.get(int(j), 0.0) + v
            for a in range(spec.nq):
                j = n_u + spec.nq * int(c) + a
                row[j] = row.get(j, 0.0) + L["B"][a, li]
            b += L["g"][li]
        rows.append(row)
        rhs.append(b)
    for c in cells_p:
        L, dm = loc[int(c)]
        rows.append({int(j): v for j, v in zip(dm, L["B"][0])})
        rhs.append(L["F"][0])
    return rows, np.array(rhs)


def test_hex128_k1_sampled_rows(vs):
    import torch
    spec = paper_element(1)
    mesh = hex_mesh(N)
    K = np.ones(mesh.n_cells)
    prob = fields.sine_problem()
    rng = np.random.default_rng(2024)
    bfaces = np.nonzero(np.asarray(mesh.face_bc) == 1)[0]
    faces = np.concatenate([rng.choice(mesh.n_faces, 48, replace=False), rng.choice(bfaces, 16, replace=False)])
    flux_rows = np.concatenate([spec.nfd * faces[:, None] + np.arange(spec.nfd)[None, :]]).ravel()
    icells = rng.choice(mesh.n_cells, 16, replace=False)
    flux_rows = np.concatenate([flux_rows, (spec.nfd * mesh.n_faces + spec.nid * icells[:, None]
                                            + np.arange(spec.nid)[None, :]).ravel()])
    cells_p = rng.choice(mesh.n_cells, 48, replace=False)
    rows, rhs = _oracle_rows(mesh, spec, K, prob, flux_rows, cells_p)
    row_ids = np.concatenate([flux_rows, spec.nfd * mesh.n_faces + spec.nid * mesh.n_cells + cells_p])

    stream = torch.cuda.current_stream().cuda_stream
    s = vs.Solver(mesh, stream=stream, device_io=1, element=vs.VEM_ELEMENT_K1, krylov=vs.VEM_KRYLOV_FGMRES,
                  restart=30, precond=vs.VEM_PREC_BLOCK_TRI, rtol=1e-8, inner_rtol=1e-8, inner_maxit=2000,
                  maxit=1000, inner=vs.VEM_INNER_AMG)
    try:
        s.set_coefficient(K)
        s.set_data(prob.f, prob.gD)
        s.assemble()
        n_u, n_p = s.sizes()
        assert (n_u, n_p) == (3 * 3 * N * N * (N + 1) + 3 * N ** 3, N ** 3)
        # 1. the assembled matrix on sampled rows
        xr = torch.from_numpy(np.random.default_rng(7).standard_normal(n_u + n_p)).cuda()
        y = torch.empty_like(xr)
        s.apply_device(xr, y)
        torch.cuda.synchronize()
        xh, yh = xr.cpu().numpy(), y.cpu().numpy()
        for r, i in zip(rows, row_ids):
            cols = np.fromiter(r.keys(), dtype=np.int64)
            vals = np.fromiter(r.values(), dtype=np.float64)
            ref = vals @ xh[cols]
            # entries agree to 1e-12 of the row's largest (the local-matrix
            # tolerance); entries that vanish exactly carry rounding noise
            tol = 1e-11 * np.abs(vals).max() * np.abs(xh[cols]).sum()
            assert abs(yh[i] - ref) <= tol, (i, yh[i], ref)
        # 2. the solve: residual of the returned solution on sampled rows
        u = torch.empty(n_u, dtype=torch.float64, device="cuda")
        p = torch.empty(n_p, dtype=torch.float64, device="cuda")
        _, _, st = s.solve(u_out=u, p_out=p)
        torch.cuda.synchronize()
    finally:
        s.close()
    assert st["relres"] <= 1e-8
    x = np.concatenate([u.cpu().numpy(), -p.cpu().numpy()])
    res = []
    for r, i, b in zip(rows, row_ids, rhs):
        cols = np.fromiter(r.keys(), dtype=np.int64)
        vals = np.fromiter(r.values(), dtype=np.float64)
        terms = np.abs(vals) @ np.abs(x[cols]) + abs(b)
        res.append(abs(b - vals @ x[cols]) / terms)
    assert max(res) <= 1e-6, max(res)
    # 3. discretisation error against the exact pressure at the centroids,
    # bounded through the pinned O(h) rate from the oracle's 8^3 solution
    m8 = hex_mesh(8)
    sys8 = assemble(m8, spec, np.ones(m8.n_cells), f=prob.f, gD=prob.gD, keep_local=True)
    _, p8 = solvers.solve_direct(sys8)
    e8 = np.abs(p8 - np.array([prob.p(c.centroid[None, :])[0] for c in sys8.cells])).max()
    cells_c = _hex_centroids(N)
    e128 = np.abs(p.cpu().numpy() - prob.p(cells_c)).max()
    assert e128 <= 2.0 * e8 * (8.0 / N), (e128, e8)


def _hex_centroids(n):
    h = 1.0 / n
    i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    return np.stack([(i.ravel() + 0.5) * h, (j.ravel() + 0.5) * h, (k.ravel() + 0.5) * h], axis=1)
