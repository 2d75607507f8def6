"""CPU FP64 oracle for the mixed virtual element method of Dassi & Scacchi,
"Parallel solvers for virtual element discretizations of elliptic equations
in mixed form" (arXiv:1901.02330).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call,
link or execute this package: only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference arm use it.  It shares no code
with the CUDA library; the only module both sides read is ``synth`` (the
seeded input generators, which hold none of the method's arithmetic).

The oracle is deliberately plain and slow: per-cell loops, dense numpy
linear algebra, numerical quadrature of high degree, ``scipy.sparse`` for
the global matrices and a direct sparse solve.  It follows the paper's
steps in its order and notation:

* Sec. 2     scaled monomials, the decomposition of vector monomials
             (Props 2.1-2.4) and the basis M^{G,+}_{k-1}      -> monomials.py
* Sec. 4.1   local velocity DOFs, face traces, divergence, the L2
             projection Pi^0_k                               -> element.py
* Sec. 4.2   pressure moments                                -> element.py
* Sec. 4.3   local forms a_{h,P}, b_{h,P}, f_{h,P}, the dofi-dofi
             stabilisation, global assembly                  -> element.py, assemble.py
* Sec. 5     block preconditioners (Block-Schur / block-triangular,
             Block-Reg), MINRES, FGMRES, Jacobi-PCG          -> solvers.py
             smoothed-aggregation AMG for S and A_reg        -> amg.py
             point-block AMG for S with several pressure
             moments per cell (k >= 2)                       -> block_amg.py
             edge-patch Schwarz smoothing for A_reg          -> schwarz.py
* Sec. 4.4   error indicators e_v, e_q                       -> errors.py

Every function is pinned by a ``-m "not gpu"`` test against something the
paper or mathematics fixes (closed forms, patch tests, table DOF counts,
conservation, convergence rates); see tests/test_oracle_*.py.
"""

from .element import ElementSpec, E0, paper_element  # noqa: F401
from .assemble import assemble, System  # noqa: F401
from . import solvers, errors, polyhedron, quadrature, monomials  # noqa: F401
