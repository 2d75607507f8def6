"""GB300 (sm_103a) solver for the mixed virtual element method of Dassi &
Scacchi (arXiv:1901.02330): element-batched assembly and block-preconditioned
Krylov solve of the saddle-point system, behind the C-ABI of
include/vemsolve.h.

The package is deliberately small:
  csrc/          CUDA kernels and the C-ABI (built into _lib/libvemsolve.so)
  build.py       in-tree nvcc build for sm_103a
  vemsolve.py    ctypes binding with the C-ABI's names (marshalling only)
  autograd.py    torch.autograd.Function over vem_solve / vem_adjoint
Importing the package does not load the library; ``vemsolve.lib()`` does,
and raises if it has not been built.
"""

__all__ = ["vemsolve", "build"]
