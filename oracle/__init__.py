"""CPU oracle for the Lindblad implicit-midpoint path -- TEST INFRASTRUCTURE.

This package is a plain, slow, obviously correct NumPy/FP64 statement of what
the GPU path computes.  It assembles dense operators (Kronecker products of
N x N matrices, the N^2 x N^2 vectorised Lindbladian) and takes every
implicit-midpoint step with a dense LU solve.  It shares no code with the CUDA
path and never imports it.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or run anything in this package; the product path
never falls back to it.

Modules
  model  -- operators, Hamiltonian, collapse operators, B-spline controls,
            dense vectorised Lindbladian (Sec. II, Appendix A).
  imr    -- implicit midpoint forward sweep, objective, discrete adjoint and
            reduced gradient (Sec. III, Appendices A-B), central differences.
  lbfgs  -- L-BFGS minimisation of G(alpha) (Sec. III; two-loop recursion of
            Nocedal & Wright), pinned by ``tests/test_oracle_lbfgs.py``.

Every function's docstring names the passage of the paper it follows.  All
functions are pinned by ``tests/test_oracle_pins.py`` against closed forms,
invariants and brute force; none is "parity unpinned".
"""

from . import model, imr, lbfgs  # noqa: F401
