"""Tolerances of the GPU parity tests, shared by the test files.

FP64: every output element within TOL64 * max|u| of the FP64 oracle.  Each
level applies operators of max norm < 2 per axis with a few dozen roundings
of 1.1e-16 per value; over <= 12 levels the drift stays near 1e-14.

FP32: within tol32(L) * max|u|, tol32(L) = 24 u (L + 1) with u = 2^-24 the
FP32 unit roundoff.  Error model: each level rounds every value a few dozen
times through operators of max norm < 2 per axis, and the coarse values carry
the error of every finer level, so the error grows with the number of levels
L + 1.  Measured on a GB300 (decomposition against the oracle, the GPU
identity, the GPU recomposition of the oracle's coefficients against the
oracle's; 1-4D, uniform and nonuniform, 27 + 7 shapes plus the 513^3 and
500x500x100 workloads): at most 5.1 u (L + 1) against the oracle and
6.8 u (L + 1) between the batched and the per-field FP32 results, so the
tolerance is 3.5-5x above the worst measured value.  Per case:
513^3 (L = 8) 1.37e-6 max|u| against tol32(8) = 1.29e-5; 500x500x100
(L = 6) 1.30e-6 against 1.00e-5; 66x64x62 (L = 5) 1.82e-6 against 8.6e-6.
"""

TOL64 = 1e-12
U32 = 2.0 ** -24


def tol32(L: int) -> float:
    """FP32 tolerance relative to max|u| for a hierarchy of L + 1 levels."""
    return 24.0 * U32 * (L + 1)
