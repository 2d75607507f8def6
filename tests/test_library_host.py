"""Host-side argument checks of the C-ABI (include/vemsolve.h): every entry
point refuses a NULL handle, vem_create refuses bad options and malformed
mesh headers with a status, and all of it happens before the library makes
its first CUDA call -- so these run without a GPU (a CUDA call here would
come back as VEM_ERR_CUDA, not VEM_ERR_BAD_INPUT)."""

import ctypes as C
import math

import numpy as np
import pytest

from synth import hex_mesh

BAD, UNSUPPORTED = 1, 8


@pytest.fixture(scope="module")
def vs():
    from paper_1901_02330_gb300 import build, vemsolve
    build.build()
    return vemsolve


def _null_args(argtypes):
    out = []
    for t in argtypes:
        if t in (C.c_int, C.c_int32, C.c_int64):
            out.append(0)
        elif t is C.c_double:
            out.append(0.0)
        else:
            out.append(None)
    return out


# entry points that take no handle, or need the device even to refuse
_NOT_HANDLE_FIRST = {"vem_default_options", "vem_create", "vem_residual_norm_noalloc",
                     "vem_launch_count", "vem_release_memory", "vem_last_error", "vem_destroy"}


def test_null_handle_is_refused_everywhere(vs):
    L = vs.lib()
    checked = 0
    for name, (res, args) in vs._SIGS.items():
        if name in _NOT_HANDLE_FIRST:
            continue
        assert args[0] is C.c_void_p, name
        st = getattr(L, name)(*_null_args(args))
        assert st == BAD, (name, st)
        checked += 1
    assert checked >= 25


def test_null_arguments_without_a_handle(vs):
    L = vs.lib()
    assert L.vem_default_options(None) == BAD
    assert L.vem_launch_count(None) == BAD
    assert L.vem_last_error(None) == b"NULL handle"
    L.vem_destroy(None)
    assert L.vem_create(None, None, None, None) == BAD
    h = C.c_void_p(1)
    assert L.vem_create(None, None, None, C.byref(h)) == BAD
    assert h.value is None                      # *out is cleared on failure
    rp = np.zeros(3, np.int64)
    assert L.vem_residual_norm_noalloc(2, None, None, None, None, None, None, None) == BAD
    assert L.vem_residual_norm_noalloc(0, rp.ctypes.data, rp.ctypes.data, rp.ctypes.data, rp.ctypes.data,
                                       rp.ctypes.data, rp.ctypes.data, None) == BAD


def test_default_options_pass_their_own_check(vs):
    """The defaults are the ones vemsolve.h documents (E0, FGMRES(30),
    block-diagonal, Jacobi-PCG to 1e-12 in at most 2000 iterations, rtol
    1e-12, maxit 2000, FP64, host I/O, reuse on, gamma = h^2) and a create
    with them gets past the option check (it then stops at the NULL mesh)."""
    o = vs.default_options()
    assert (o.element, o.krylov, o.restart, o.precond, o.inner, o.precision) == (
        vs.VEM_ELEMENT_E0, vs.VEM_KRYLOV_FGMRES, 30, vs.VEM_PREC_BLOCK_DIAG, vs.VEM_INNER_PCG,
        vs.VEM_PRECISION_FP64)
    assert (o.rtol, o.maxit, o.inner_rtol, o.inner_maxit) == (1e-12, 2000, 1e-12, 2000)
    assert (o.device_io, o.reuse, o.reg_gamma) == (0, 1, 0.0)
    h = C.c_void_p()
    assert vs.lib().vem_create(None, C.byref(o), None, C.byref(h)) == BAD and not h.value


BAD_OPTIONS = {
    "element": dict(element=3),
    "krylov": dict(krylov=2),
    "precond": dict(precond=3),
    "minres-tri": dict(krylov=0, precond=1),
    "reg_gamma<0": dict(reg_gamma=-1.0),
    "reg_gamma-nan": dict(reg_gamma=math.nan),
    "reg_gamma-inf": dict(reg_gamma=math.inf),
    "inner": dict(inner=3),
    "precision": dict(precision=2),
    "inner_smoother": dict(inner_smoother=2),
    "inner_smoother<0": dict(inner_smoother=-1),
    "reg_cycle": dict(reg_cycle=2),
    "mixed-minres": dict(precision=1, krylov=0, precond=0),
    "restart0": dict(restart=0),
    "restart257": dict(restart=257),
    "reuse": dict(reuse=2),
    "rtol0": dict(rtol=0.0),
    "inner_rtol-nan": dict(inner_rtol=math.nan),
    "maxit0": dict(maxit=0),
    "inner_maxit0": dict(inner_maxit=0),
}


@pytest.mark.parametrize("name", list(BAD_OPTIONS))
def test_bad_options_refused_before_the_device(vs, name):
    with pytest.raises(vs.VemError) as e:
        vs.Solver(hex_mesh(2), **BAD_OPTIONS[name])
    assert e.value.code == BAD


def _mesh_struct(vs, arrays, n_vertices=None, n_faces=None, n_cells=None):
    xyz, fvp, fv, cfp, cf, fbc = arrays
    return vs.vem_mesh(xyz.shape[0] if n_vertices is None else n_vertices, xyz.ctypes.data,
                       fvp.shape[0] - 1 if n_faces is None else n_faces, fvp.ctypes.data, fv.ctypes.data,
                       cfp.shape[0] - 1 if n_cells is None else n_cells, cfp.ctypes.data, cf.ctypes.data,
                       fbc.ctypes.data)


def _arrays(m):
    return [np.ascontiguousarray(m.xyz, np.float64), np.ascontiguousarray(m.face_vtx_ptr, np.int64),
            np.ascontiguousarray(m.face_vtx, np.int32), np.ascontiguousarray(m.cell_face_ptr, np.int64),
            np.ascontiguousarray(m.cell_face, np.int32), np.ascontiguousarray(m.face_bc, np.int8)]


def _create(vs, mesh_struct):
    h = C.c_void_p()
    o = vs.default_options()
    st = vs.lib().vem_create(C.byref(mesh_struct), C.byref(o), None, C.byref(h))
    assert not h.value
    return st


def test_malformed_mesh_headers_refused_before_the_device(vs):
    m = hex_mesh(2)
    a = _arrays(m)
    # counts
    assert _create(vs, _mesh_struct(vs, a, n_cells=0)) == BAD
    assert _create(vs, _mesh_struct(vs, a, n_faces=3)) == BAD
    assert _create(vs, _mesh_struct(vs, a, n_vertices=3)) == BAD
    assert _create(vs, _mesh_struct(vs, a, n_faces=2 ** 31, n_cells=1)) == UNSUPPORTED
    # CSR pointers that do not start at 0
    b = [x.copy() for x in a]
    b[1][0] = 1
    assert _create(vs, _mesh_struct(vs, b)) == BAD
    b = [x.copy() for x in a]
    b[3][0] = 2
    assert _create(vs, _mesh_struct(vs, b)) == BAD
    # totals outside [3, 4096] vertices per face and [4, 256] faces per cell
    b = [x.copy() for x in a]
    b[1][-1] = 2 * (b[1].shape[0] - 1)
    assert _create(vs, _mesh_struct(vs, b)) == BAD
    b = [x.copy() for x in a]
    b[3][-1] = 3 * (b[3].shape[0] - 1)
    assert _create(vs, _mesh_struct(vs, b)) == BAD
    b = [x.copy() for x in a]
    b[3][-1] = 257 * (b[3].shape[0] - 1)
    assert _create(vs, _mesh_struct(vs, b)) == BAD
    # a NULL array
    s = _mesh_struct(vs, a)
    s.face_bc = None
    assert _create(vs, s) == BAD
