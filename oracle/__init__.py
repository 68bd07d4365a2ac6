"""FP64 CPU oracle for the 7-point stencil BiCGStab path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product library imports, links or
executes this package; only the tests, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.  It shares
no code with the CUDA path: it is plain NumPy in float64, written from the
paper (Fan et al., "Fast Stencil-Code Computation on a Wafer-Scale
Processor", SC20) and from the mathematics of the operator.

Modules
-------
``stencil``   the operator ``(A v)_i`` (Sec. IV-A), Jacobi scaling to a unit
              diagonal (Sec. IV), rounding to storage types, dense assembly
              and an independently built transpose.
``bicgstab``  Algorithm 1 (standard BiCGStab) step by step, with the stopping
              rule, start vector and breakdown readings of the project.
``direct``    exact small-mesh solvers used as pins: dense LU (LAPACK),
              conjugate gradients, the Thomas tridiagonal algorithm, and the
              closed-form Dirichlet-Laplacian eigenpairs.
``counts``    the paper's operation count per mesh point (Table I) and the
              byte model of one fused iteration.
``fp32model`` Algorithm 1 under a float32 rounding model with a chosen
              summation order: bounds the step count of a float32 solve
              (a model of rounding, not a reference for values).

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against closed forms, brute force or a library routine (see ``tests/``),
except where a function's docstring says "parity unpinned".
"""

from . import counts, direct, stencil, bicgstab, fp32model  # noqa: F401
