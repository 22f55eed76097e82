"""CPU FP64 oracle for the localizing gradient damage method (LGDM).

TEST INFRASTRUCTURE ONLY.  This package is the independent, slow, plain
statement of what the GPU path computes; it exists so that tests, the smoke
check and the benchmark's CPU-baseline leg can compare against it.  The
product path (the CUDA library and its Python binding) never imports it, and
it imports nothing from the product path: the only code both sides share is
the seeded input generator ``lgdm_inputs``, which holds no method arithmetic.

Contents, in the paper's order:
  constitutive.py  damage law (Eq. A.1), history (Eq. A.2), modified von Mises
                   equivalent strain (Eq. A.3), interaction function (Eq. A.4),
                   isotropic elasticity, free energy (Eq. 1)
  element.py       Gauss-point integration of the coupled element tangent
                   (Eq. 11a-d) and residual (Eq. 11e-f), vectorised over
                   elements like the paper's Algorithm 2
  assembly.py      global sparse assembly (the paper's triplet ``sparse``
                   assembly), Dirichlet handling, reaction
  newton.py        incremental-iterative Newton driver (Algorithm 2) with a
                   direct sparse solve, history commit, energy bookkeeping

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed forms, complex-step derivatives, patch tests, brute-force assembly,
the elastic-bar closed form, invariants).  The full load-displacement curves
have no printed values to pin against (the paper's curves are figures), so the
Newton driver is pinned only through its parts and the invariants listed in
tests/test_oracle_pins.py.
"""
from . import constitutive, element, assembly, newton  # noqa: F401
