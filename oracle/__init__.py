"""FP64 CPU oracle for quantics tensor-train arithmetic.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import or run anything in this
package.  The library (``paper_2602_20226_gb300``) never imports it and shares no
code with it; the only common module is the seeded input generator
``paper_2602_20226_gb300.inputs``, which holds no tensor-train arithmetic.

Modules
  core        exact apply / hadamard / add / inner / evaluate, orthogonalisation,
              rounding, gauge-invariant error e(a, b)            (Sections 2, 3.1, 3.2)
  structured  closed-form exp / cos / sin / polynomial TTs, shift MPOs and
              Dirichlet Laplacians                              (Section 4)
  grad        hand-derived adjoints of apply / hadamard / inner / evaluate / rounding
  approx      the decomposition (zip-up) and variational approximations of W x
                                                                 (Sections 3.2, 3.3)
  qft         the Fourier (DFT) matrix as a tensor train from element-wise products of
              rank-b_q factors, rounded at a maximum rank            (Section 4.3)

Every function is pinned by ``tests/test_oracle_*.py`` against brute force on
full tensors, closed forms, invariants or finite differences.
"""
from . import approx, core, grad, qft, structured  # noqa: F401
