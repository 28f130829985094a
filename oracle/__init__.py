"""FP64 CPU oracle for the extra-component method -- TEST INFRASTRUCTURE ONLY.

This package is a plain, slow, deliberately unoptimised restatement of the
paper's method (Terekhov, "An extra-component method for evaluating fast
matrix-vector multiplication with special functions"), used to check the CUDA
path.  It shares no code with the CUDA library: no kernels, headers, tables,
constants or helpers.  Only the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference arm of ``bench.py`` may import it; the product path
never does.

Modules
-------
special   Kaiser window, I0, the Newton solve for zeta(eps1), the extra-component
          count s(eps2, zeta), FFT-friendly lengths and the block schedule
          (Section 2.2, Algorithms 1-4, Section 3).
families  Nodes, quadrature weights and matrix entries of the special-function
          families by three-term recurrence (Sections 2.1, 3, 4).
method    The compressed matrices and the apply / adjoint apply
          (eqs. (comp1), (comp2), (Fe1), (Fe2), (Fe3); Algorithms 1-4),
          plus the plain dense products that define the result.
method2d  The two-dimensional compression F W D W F (eq. (comp_2d)) and its
          block scheme (Sections 4.2, 5.3) for Laguerre / Hermite functions
          at equispaced nodes and the index kernels A^[1], A^[2].

Parity status: every function is pinned by a test in tests/test_oracle_*.py
except where its docstring says "parity unpinned".  Parity unpinned: the
compression ratio (kept elements per row) of Laguerre functions at
Gauss-Laguerre nodes and Hermite functions at Gauss-Hermite nodes, for which
the paper prints no numbers (reported, not pinned).
"""
from . import special, families, method, method2d  # noqa: F401
