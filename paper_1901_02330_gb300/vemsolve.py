"""Thin ctypes binding of include/vemsolve.h (argument marshalling only).

Every computation runs in the CUDA library ``_lib/libvemsolve.so``; this
module converts numpy arrays / torch tensors to pointers and status codes to
exceptions.  It fails loudly when the library is missing: there is no CPU
fallback.
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libvemsolve.so")

VEM_OK = 0
STATUS = {0: "VEM_OK", 1: "VEM_ERR_BAD_INPUT", 2: "VEM_ERR_DEGENERATE_MESH", 3: "VEM_ERR_NOT_CONVERGED",
          4: "VEM_ERR_BREAKDOWN", 5: "VEM_ERR_NONFINITE", 6: "VEM_ERR_OOM", 7: "VEM_ERR_CUDA",
          8: "VEM_ERR_UNSUPPORTED"}
VEM_ELEMENT_E0, VEM_ELEMENT_K1, VEM_ELEMENT_K2 = 0, 1, 2
VEM_KRYLOV_MINRES, VEM_KRYLOV_FGMRES = 0, 1
VEM_PREC_BLOCK_DIAG, VEM_PREC_BLOCK_TRI, VEM_PREC_BLOCK_REG = 0, 1, 2
VEM_AMG_SCHUR, VEM_AMG_REG = 0, 1
VEM_INNER_PCG, VEM_INNER_AMG, VEM_INNER_BLOCK_AMG = 0, 1, 2
VEM_PRECISION_FP64, VEM_PRECISION_MIXED = 0, 1
VEM_SMOOTH_JACOBI, VEM_SMOOTH_CHEBYSHEV = 0, 1
VEM_REG_SCALAR_AMG, VEM_REG_CONDENSED = 0, 1
VEM_QP_CELL, VEM_QP_BFACE = 0, 1


class vem_mesh(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("xyz", C.c_void_p),
                ("n_faces", C.c_int64), ("face_vtx_ptr", C.c_void_p), ("face_vtx", C.c_void_p),
                ("n_cells", C.c_int64), ("cell_face_ptr", C.c_void_p), ("cell_face", C.c_void_p),
                ("face_bc", C.c_void_p)]


class vem_options(C.Structure):
    _fields_ = [("element", C.c_int), ("krylov", C.c_int), ("restart", C.c_int), ("rtol", C.c_double),
                ("maxit", C.c_int), ("precond", C.c_int), ("inner", C.c_int), ("inner_rtol", C.c_double),
                ("inner_maxit", C.c_int), ("precision", C.c_int), ("device_io", C.c_int), ("reuse", C.c_int),
                ("reg_gamma", C.c_double), ("inner_smoother", C.c_int), ("reg_cycle", C.c_int)]


class vem_stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("inner_iterations", C.c_int32), ("relres", C.c_double),
                ("t_assemble_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("n_u", C.c_int64), ("n_p", C.c_int64), ("nnz_A", C.c_int64), ("nnz_S", C.c_int64),
                ("t_element_ms", C.c_double), ("t_scatter_ms", C.c_double), ("n_classes", C.c_int64),
                ("t_schur_spmv_ms", C.c_double), ("n_schur_spmv", C.c_int64),
                ("t_amg_setup_ms", C.c_double), ("amg_levels", C.c_int32),
                ("t_saddle_spmv_ms", C.c_double), ("n_saddle_spmv", C.c_int64),
                ("multiplier", C.c_double), ("schur_tile", C.c_int32),
                ("reg_gamma", C.c_double), ("nnz_reg", C.c_int64),
                ("t_vc_resid_ms", C.c_double), ("n_vc_resid", C.c_int64),
                ("t_vc_post_ms", C.c_double), ("n_vc_post", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class VemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None

# name -> (restype, argtypes); the exported C-ABI, one entry per declaration
_SIGS = {
    "vem_default_options": (C.c_int, [C.POINTER(vem_options)]),
    "vem_create": (C.c_int, [C.POINTER(vem_mesh), C.POINTER(vem_options), C.c_void_p, C.POINTER(C.c_void_p)]),
    "vem_set_options": (C.c_int, [C.c_void_p, C.POINTER(vem_options)]),
    "vem_sizes": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "vem_quadrature_count": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int64)]),
    "vem_quadrature_points": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "vem_set_coefficient": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vem_set_source": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vem_set_coefficient_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vem_set_log_coefficient_device": (C.c_int, [C.c_void_p, C.c_void_p]),
    "vem_set_source_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vem_assemble": (C.c_int, [C.c_void_p]),
    "vem_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(vem_stats)]),
    "vem_solve_batched": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.POINTER(vem_stats)]),
    "vem_adjoint": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(vem_stats)]),
    "vem_get_geometry": (C.c_int, [C.c_void_p] + [C.c_void_p] * 7),
    "vem_local_size": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "vem_get_local": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vem_assemble_local": (C.c_int, [C.c_void_p]),
    "vem_local_time": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
    "vem_get_system": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vem_get_schur": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "vem_apply_device": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vem_residual_norm_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_void_p]),
    "vem_bface_info": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "vem_amg_setup": (C.c_int, [C.c_void_p, C.c_int32]),
    "vem_amg_levels": (C.c_int, [C.c_void_p, C.c_int32, C.POINTER(C.c_int32), C.c_void_p, C.c_void_p,
                                 C.c_void_p]),
    "vem_amg_get_level": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32] + [C.c_void_p] * 7),
    "vem_amg_vcycle_device": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]),
    "vem_launch_count": (C.c_int, [C.POINTER(C.c_int64)]),
    "vem_last_error": (C.c_char_p, [C.c_void_p]),
    "vem_destroy": (None, [C.c_void_p]),
    "vem_release_memory": (C.c_int, []),
}


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {_LIB_PATH} is missing "
                               "(run python -m paper_1901_02330_gb300.build)")
        L = C.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def launch_count() -> int:
    n = C.c_int64()
    lib().vem_launch_count(C.byref(n))
    return n.value


def release_memory() -> None:
    """Return the unused part of the library's device memory pool (and its
    cached pinned host buffers) to the system."""
    st = lib().vem_release_memory()
    if st != VEM_OK:
        raise VemError(st, "vem_release_memory")


def residual_norm_noalloc(row_ptr, col, val, x, b, out, stream: int = 0) -> None:
    """vem_residual_norm_noalloc on device tensors: out[0] = ||b - A x||,
    out[1] = ||b||, out[2] = their ratio.  Allocates nothing on the device
    (for callers whose device memory is owned by another allocator); the
    result is ready when the stream reaches it.

    The library reads the buffers through raw device pointers, so every
    argument is checked here first: contiguous CUDA tensors on the current
    device, row_ptr int64 with rows + 1 entries, col int32, val / x / b / out
    float64, val and col holding row_ptr[-1] entries, x and b rows entries
    (the matrix is square) and out at least 3.  Column ids must lie in
    [0, rows); they are not scanned here (that would need device memory)."""
    import torch
    args = dict(row_ptr=row_ptr, col=col, val=val, x=x, b=b, out=out)
    want = dict(row_ptr=torch.int64, col=torch.int32, val=torch.float64, x=torch.float64, b=torch.float64,
                out=torch.float64)
    for k, t in args.items():
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{k}: a torch CUDA tensor is required, got {type(t).__name__}")
    dev = torch.cuda.current_device() if torch.cuda.is_available() else -1
    for k, t in args.items():
        if t.device.type != "cuda" or t.device.index != dev:
            raise ValueError(f"{k}: must be on the current CUDA device cuda:{dev}, is on {t.device}")
        if t.dtype != want[k]:
            raise TypeError(f"{k}: dtype {want[k]} required, got {t.dtype}")
        if not t.is_contiguous() or t.dim() != 1:
            raise ValueError(f"{k}: a contiguous 1-D tensor is required")
    rows = int(row_ptr.numel()) - 1
    if rows < 1:
        raise ValueError("row_ptr: needs at least 2 entries")
    nnz = int(row_ptr[-1].item())
    if int(row_ptr[0].item()) != 0 or nnz < 0:
        raise ValueError("row_ptr: must start at 0 and end at the entry count")
    if col.numel() < nnz or val.numel() < nnz:
        raise ValueError(f"col / val: {nnz} entries required, have {col.numel()} / {val.numel()}")
    if x.numel() != rows or b.numel() != rows:
        raise ValueError(f"x / b: {rows} entries required, have {x.numel()} / {b.numel()}")
    if out.numel() < 3:
        raise ValueError("out: at least 3 entries required")
    st = lib().vem_residual_norm_noalloc(rows, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(x), _ptr(b),
                                         _ptr(out), C.c_void_p(stream or None))
    if st != VEM_OK:
        raise VemError(st, "vem_residual_norm_noalloc")


def library_path() -> str:
    return _LIB_PATH


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return a.data_ptr()
    raise TypeError(type(a))


def default_options(**kw) -> vem_options:
    o = vem_options()
    lib().vem_default_options(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Solver:
    """One vem_handle.  ``mesh`` has the synth.Mesh fields; stream is a
    cudaStream_t as an int (e.g. torch.cuda.current_stream().cuda_stream)."""

    def __init__(self, mesh, options: vem_options | None = None, stream: int = 0, **kw):
        self._h = C.c_void_p()
        self._keep = [np.ascontiguousarray(mesh.xyz, dtype=np.float64),
                      np.ascontiguousarray(mesh.face_vtx_ptr, dtype=np.int64),
                      np.ascontiguousarray(mesh.face_vtx, dtype=np.int32),
                      np.ascontiguousarray(mesh.cell_face_ptr, dtype=np.int64),
                      np.ascontiguousarray(mesh.cell_face, dtype=np.int32),
                      np.ascontiguousarray(mesh.face_bc, dtype=np.int8)]
        xyz, fvp, fv, cfp, cf, fbc = self._keep
        m = vem_mesh(xyz.shape[0], _ptr(xyz), fvp.shape[0] - 1, _ptr(fvp), _ptr(fv),
                     cfp.shape[0] - 1, _ptr(cfp), _ptr(cf), _ptr(fbc))
        self.options = options if options is not None else default_options(**kw)
        st = lib().vem_create(C.byref(m), C.byref(self.options), C.c_void_p(stream or None), C.byref(self._h))
        if st != VEM_OK:
            raise VemError(st, "vem_create failed")
        self.n_faces = int(fvp.shape[0] - 1)
        self.n_cells = int(cfp.shape[0] - 1)
        self.cell_face_ptr = cfp.copy()
        self.generation = 0          # counts solves (the adjoint uses the latest)

    # -- status handling
    def _check(self, st, what=""):
        if st != VEM_OK:
            msg = lib().vem_last_error(self._h)
            raise VemError(st, (msg.decode() if msg else "") or what)

    def close(self):
        if self._h:
            lib().vem_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- C-ABI calls
    def set_options(self, **kw):
        for k, v in kw.items():
            setattr(self.options, k, v)
        self._check(lib().vem_set_options(self._h, C.byref(self.options)))

    def sizes(self):
        nu, np_ = C.c_int64(), C.c_int64()
        self._check(lib().vem_sizes(self._h, C.byref(nu), C.byref(np_)))
        return nu.value, np_.value

    def quadrature_count(self, which: int) -> int:
        n = C.c_int64()
        self._check(lib().vem_quadrature_count(self._h, which, C.byref(n)))
        return n.value

    def quadrature_points(self, which: int, out=None):
        """[n, 3] coordinates; into out when given (numpy, or a contiguous
        float64 CUDA tensor on the handle's device)."""
        n = self.quadrature_count(which)
        if out is None:
            out = np.zeros((n, 3))
        elif tuple(out.shape) != (n, 3):
            raise ValueError(f"out must have shape ({n}, 3)")
        elif hasattr(out, "data_ptr"):
            import torch
            if out.dtype != torch.float64 or not out.is_contiguous():
                raise ValueError("out must be a contiguous float64 tensor")
        elif out.dtype != np.float64 or not out.flags.c_contiguous:
            raise ValueError("out must be a C-contiguous float64 array")
        if n:
            self._check(lib().vem_quadrature_points(self._h, which, _ptr(out)))
        return out

    def set_coefficient(self, K):
        if hasattr(K, "data_ptr"):
            self._check(lib().vem_set_coefficient_device(self._h, _ptr(K)))
        else:
            K = np.ascontiguousarray(K, dtype=np.float64)
            assert K.shape == (self.n_cells,)
            self._check(lib().vem_set_coefficient(self._h, _ptr(K)))

    def set_log_coefficient(self, logK):
        """theta = log K per cell as a CUDA float64 tensor (vem_set_log_coefficient_device)."""
        if not hasattr(logK, "data_ptr") or logK.device.type != "cuda" or logK.dtype.itemsize != 8:
            raise TypeError("log K: a CUDA float64 tensor is required")
        if logK.numel() != self.n_cells:
            raise ValueError(f"log K: {self.n_cells} entries required, have {logK.numel()}")
        self._check(lib().vem_set_log_coefficient_device(self._h, _ptr(logK)))

    def set_source(self, f_qp=None, gD_qp=None):
        dev = any(hasattr(a, "data_ptr") for a in (f_qp, gD_qp) if a is not None)
        if dev:
            self._check(lib().vem_set_source_device(self._h, _ptr(f_qp), _ptr(gD_qp)))
        else:
            f = None if f_qp is None else np.ascontiguousarray(f_qp, dtype=np.float64)
            g = None if gD_qp is None else np.ascontiguousarray(gD_qp, dtype=np.float64)
            self._check(lib().vem_set_source(self._h, _ptr(f), _ptr(g)))

    def bface_info(self):
        """(outward unit normals [n][3], face flags [n]) at the boundary points."""
        n = C.c_int64()
        self._check(lib().vem_quadrature_count(self._h, VEM_QP_BFACE, C.byref(n)))
        nrm = np.zeros((n.value, 3))
        flg = np.zeros(n.value, dtype=np.int8)
        if n.value:
            self._check(lib().vem_bface_info(self._h, _ptr(nrm), _ptr(flg)))
        return nrm, flg

    def set_data(self, f=None, gD=None, flux=None):
        """Evaluate callables at the library's quadrature points: f at the cell
        points, g_D on Dirichlet faces and u.n_out of the vector field flux on
        prescribed-flux faces."""
        fq = f(self.quadrature_points(VEM_QP_CELL)) if f is not None else None
        pb = self.quadrature_points(VEM_QP_BFACE)
        gq = None
        if pb.shape[0] and (gD is not None or flux is not None):
            nrm, flg = self.bface_info()
            gq = np.zeros(pb.shape[0])
            if gD is not None and np.any(flg == 1):
                gq[flg == 1] = gD(pb[flg == 1])
            if flux is not None and np.any(flg == 2):
                gq[flg == 2] = np.einsum("ij,ij->i", flux(pb[flg == 2]), nrm[flg == 2])
        self.set_source(fq, gq)

    def assemble(self):
        self._check(lib().vem_assemble(self._h))

    def solve(self, x0=None, u_out=None, p_out=None, allow_not_converged=False):
        """Host I/O (numpy) unless options.device_io, then torch/device arrays."""
        nu, np_ = self.sizes()
        if u_out is None:
            u_out = np.zeros(nu)
        if p_out is None:
            p_out = np.zeros(np_)
        st = vem_stats()
        x0p = None
        if x0 is not None:
            x0 = x0 if hasattr(x0, "data_ptr") else np.ascontiguousarray(x0, dtype=np.float64)
            x0p = _ptr(x0)
        code = lib().vem_solve(self._h, x0p, _ptr(u_out), _ptr(p_out), C.byref(st))
        self.generation += 1
        if not (code == 3 and allow_not_converged):
            self._check(code)
        return u_out, p_out, st.as_dict()

    def solve_batched(self, K, f_qp=None, gD_qp=None, u_out=None, p_out=None, allow_not_converged=False):
        """K, f_qp, gD_qp with a leading batch axis; host numpy unless device_io."""
        nb = int(K.shape[0])
        nu, np_ = self.sizes()
        dev = bool(self.options.device_io)
        # the library reads nb rows of these sizes: refuse anything shorter
        want = {"K": (K, self.n_cells), "f_qp": (f_qp, self.quadrature_count(VEM_QP_CELL)),
                "gD_qp": (gD_qp, self.quadrature_count(VEM_QP_BFACE))}
        for name, (arr, m) in want.items():
            if arr is not None and tuple(arr.shape) != (nb, m):
                raise ValueError(f"{name} must have shape ({nb}, {m}), not {tuple(arr.shape)}")
        if not dev:
            K = np.ascontiguousarray(K, dtype=np.float64)
            f_qp = None if f_qp is None else np.ascontiguousarray(f_qp, dtype=np.float64)
            gD_qp = None if gD_qp is None else np.ascontiguousarray(gD_qp, dtype=np.float64)
            if u_out is None:
                u_out = np.zeros((nb, nu))
            if p_out is None:
                p_out = np.zeros((nb, np_))
        rel = np.zeros(nb)
        st = vem_stats()
        code = lib().vem_solve_batched(self._h, nb, _ptr(K), _ptr(f_qp), _ptr(gD_qp), _ptr(u_out), _ptr(p_out),
                                       _ptr(rel), C.byref(st))
        self.generation += 1
        if not (code == 3 and allow_not_converged):
            self._check(code)
        return u_out, p_out, rel, st.as_dict()

    def adjoint(self, dL_du=None, dL_dp=None, out=None):
        """dL/dlog K per cell for the last solve (host numpy unless device_io)."""
        if out is None:
            out = np.zeros(self.n_cells)
        if not self.options.device_io:
            dL_du = None if dL_du is None else np.ascontiguousarray(dL_du, dtype=np.float64)
            dL_dp = None if dL_dp is None else np.ascontiguousarray(dL_dp, dtype=np.float64)
        st = vem_stats()
        self._check(lib().vem_adjoint(self._h, _ptr(dL_du), _ptr(dL_dp), _ptr(out), C.byref(st)))
        return out, st.as_dict()

    def geometry(self):
        nf, nc = self.n_faces, self.n_cells
        out = dict(face_area=np.zeros(nf), face_centroid=np.zeros((nf, 3)), face_normal=np.zeros((nf, 3)),
                   face_diam=np.zeros(nf), cell_volume=np.zeros(nc), cell_centroid=np.zeros((nc, 3)),
                   cell_diam=np.zeros(nc))
        self._check(lib().vem_get_geometry(self._h, *[_ptr(out[k]) for k in
                                                      ("face_area", "face_centroid", "face_normal", "face_diam",
                                                       "cell_volume", "cell_centroid", "cell_diam")]))
        return out

    def local_matrices(self):
        """List of (M_P, B_P) per cell in the cell's local DOF order."""
        mt, bt = C.c_int64(), C.c_int64()
        self._check(lib().vem_local_size(self._h, C.byref(mt), C.byref(bt)))
        M = np.zeros(mt.value)
        off = np.zeros(self.n_cells + 1, dtype=np.int64)
        B = np.zeros(bt.value)
        self._check(lib().vem_get_local(self._h, _ptr(M), _ptr(off), _ptr(B)))
        nfd, nid, nq = {VEM_ELEMENT_E0: (1, 0, 1), VEM_ELEMENT_K1: (3, 3, 1),
                        VEM_ELEMENT_K2: (6, 14, 4)}[self.options.element]
        out = []
        for c in range(self.n_cells):
            k = int(self.cell_face_ptr[c + 1] - self.cell_face_ptr[c])
            nl = nfd * k + nid
            b0 = nq * (nfd * int(self.cell_face_ptr[c]) + nid * c)
            Bc = B[b0:b0 + nq * nl]
            out.append((M[off[c]:off[c] + nl * nl].reshape(nl, nl), Bc if nq == 1 else Bc.reshape(nq, nl)))
        return out

    def assemble_local(self):
        """Element matrices only (vem_assemble_local); returns (element kernel
        ms, classes evaluated)."""
        self._check(lib().vem_assemble_local(self._h))
        ms, nc = C.c_double(), C.c_int64()
        self._check(lib().vem_local_time(self._h, C.byref(ms), C.byref(nc)))
        return ms.value, nc.value

    def system(self):
        """(A as scipy CSR [M B^T; B 0], rhs [g; F])."""
        import scipy.sparse as sp
        nu, np_ = self.sizes()
        n = nu + np_
        rp = np.zeros(n + 1, dtype=np.int64)
        self._check(lib().vem_get_system(self._h, _ptr(rp), None, None, None))
        col = np.zeros(rp[-1], dtype=np.int32)
        val = np.zeros(rp[-1])
        rhs = np.zeros(n)
        self._check(lib().vem_get_system(self._h, _ptr(rp), _ptr(col), _ptr(val), _ptr(rhs)))
        return sp.csr_matrix((val, col, rp), shape=(n, n)), rhs

    def schur(self):
        import scipy.sparse as sp
        nu, np_ = self.sizes()
        rp = np.zeros(np_ + 1, dtype=np.int64)
        self._check(lib().vem_get_schur(self._h, _ptr(rp), None, None, None))
        col = np.zeros(rp[-1], dtype=np.int32)
        val = np.zeros(rp[-1])
        dM = np.zeros(nu)
        self._check(lib().vem_get_schur(self._h, _ptr(rp), _ptr(col), _ptr(val), _ptr(dM)))
        return sp.csr_matrix((val, col, rp), shape=(np_, np_)), dM

    # -- AMG hierarchies: of S (VEM_INNER_AMG) or of A_reg (Block-Reg)
    def amg_setup(self, which=VEM_AMG_SCHUR):
        self._check(lib().vem_amg_setup(self._h, which))

    def amg_levels(self, which=VEM_AMG_SCHUR):
        """(rows, nnz, nnz of P) per level."""
        nl = C.c_int32()
        rows = np.zeros(16, dtype=np.int64)
        nnz = np.zeros(16, dtype=np.int64)
        nnzp = np.zeros(16, dtype=np.int64)
        self._check(lib().vem_amg_levels(self._h, which, C.byref(nl), _ptr(rows), _ptr(nnz), _ptr(nnzp)))
        k = nl.value
        return rows[:k].copy(), nnz[:k].copy(), nnzp[:k].copy()

    def amg_level(self, level: int, which=VEM_AMG_SCHUR):
        """(A_l as scipy CSR, agg or None, P_l as scipy CSR or None)."""
        import scipy.sparse as sp
        rows, nnz, nnzp = self.amg_levels(which)
        n = int(rows[level])
        rp = np.zeros(n + 1, dtype=np.int64)
        col = np.zeros(max(int(nnz[level]), 1), dtype=np.int32)
        val = np.zeros(max(int(nnz[level]), 1))
        coarse = level + 1 < rows.size
        agg = np.zeros(n, dtype=np.int32) if coarse else None
        prp = np.zeros(n + 1, dtype=np.int64) if coarse else None
        pcol = np.zeros(max(int(nnzp[level]), 1), dtype=np.int32) if coarse else None
        pval = np.zeros(max(int(nnzp[level]), 1)) if coarse else None
        self._check(lib().vem_amg_get_level(self._h, which, level, _ptr(rp), _ptr(col), _ptr(val), _ptr(agg),
                                            _ptr(prp), _ptr(pcol), _ptr(pval)))
        A = sp.csr_matrix((val[:rp[-1]], col[:rp[-1]], rp), shape=(n, n))
        P = None
        if coarse:
            P = sp.csr_matrix((pval[:prp[-1]], pcol[:prp[-1]], prp), shape=(n, int(rows[level + 1])))
        return A, agg, P

    def amg_vcycle_device(self, b, x, which=VEM_AMG_SCHUR):
        self._check(lib().vem_amg_vcycle_device(self._h, which, _ptr(b), _ptr(x)))

    def apply_device(self, x, y):
        self._check(lib().vem_apply_device(self._h, _ptr(x), _ptr(y)))
