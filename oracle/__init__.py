"""CPU FP64 oracle for FLAPW H/S assembly, the matching coefficients A, B the
assembly takes as inputs, and the reduction of the generalized eigenproblem
H c = lambda S c that H and S define.

TEST INFRASTRUCTURE: only tests, the smoke check and the CPU-baseline leg of
the benchmark may import this package.  It shares no code with the CUDA
library, and the library never calls it.

Parity status: every function here is pinned: ``tests/test_oracle_pins.py`` (exact
brute force, closed forms, invariants, textbook Cholesky checks) and
``tests/test_oracle_matching.py`` (the matching conditions rebuild the plane wave and
its radial derivative on the sphere; spherical harmonics against closed forms and
orthonormality).
"""
from .hs_oracle import assemble, h_aa, rel_frobenius  # noqa: F401
from .cholesky import cholesky_lower, fail_flags  # noqa: F401
from .reduce import reduce_standard, standard_eigenvalues  # noqa: F401
