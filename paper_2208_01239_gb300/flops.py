"""Real-flop counts (coefficient of n^3, leading order) used for reporting.

Two conventions are kept apart:

* ``paper_*`` -- the counts stated in Sec. 4.1 (Proposition "Flop counts":
  28/3 for Frobenius inversion with LU, 32/3 for complex LU inversion) and
  Sec. 4.3 (23/3 for Frobenius inversion with Cholesky, 28/3 for complex
  Cholesky inversion).  The paper counts a complex flop as four real flops
  (proof of Theorem "threshold") and does not exploit the zero structure of the
  identity right-hand side.
* ``executed_*`` -- the work the CUDA path actually performs, stage by stage
  (zero blocks of triangular right-hand sides are skipped, the symmetric
  product X1^T X1 forms the lower triangle only, the inverse of a Cholesky
  factor's Gram matrix, L^{-T} L^{-1}, is the product of the triangular
  inverse with itself over k >= max(i, j), as LAPACK's potri, forming the
  tiles on and below the diagonal only, since such a product is symmetric /
  Hermitian in floating point too).

``nominal`` = 8 n^3 is the same for every method, so that TFLOP/s figures are
comparable the way inversions/s are.
"""
from __future__ import annotations

from fractions import Fraction as F

# Sec. 4.1 and 4.3, leading-order coefficients of n^3
PAPER = {
    "frob_lu": F(2, 3) + 2 + 2 + F(2, 3) + 4,          # LU, solve, mult+add, LU, 2n right solves
    "cplx_lu": 4 * (F(2, 3) + 1 + 1),                 # complex LU + 2 substitutions with I
    "frob_chol": F(2, 3) + 2 + 2 + 1 + 2,             # 2 Cholesky, 2n back + 2n fwd subs, SYRK, GEMM
    "cplx_chol": 4 * (F(1, 3) + 1 + 1),               # complex Cholesky + 2 substitutions with I
}

# What the CUDA path executes (stage list in the same order as the kernels run)
EXECUTED_STAGES = {
    "frob_lu": [("getrf A", F(2, 3)), ("L1 U1 X1 = P1 B", F(2)), ("S = A + B X1", F(2)),
                ("getrf S", F(2, 3)), ("S^{-1} from L2 U2", F(4, 3)), ("X1 S^{-1}", F(2))],
    "cplx_lu": [("zgetrf", 4 * F(2, 3)), ("z U^{-1} L^{-1} P", 4 * F(4, 3))],
    "frob_chol": [("potrf A", F(1, 3)), ("R1^T X1 = B", F(1)), ("S = A - X1^T X1 (lower)", F(1)),
                  ("R1 X2 = X1", F(1)), ("potrf S", F(1, 3)), ("R2^T X5 = I", F(1, 3)),
                  ("X6 = X5^T X5 (lower)", F(1, 3)), ("X2 X6", F(2))],
    "cplx_chol": [("zpotrf", 4 * F(1, 3)), ("R^H X1 = I", 4 * F(1, 3)), ("X2 = X1^H X1 (lower)", 4 * F(1, 3))],
}
EXECUTED = {k: sum(c for _, c in v) for k, v in EXECUTED_STAGES.items()}

NOMINAL = F(8)


def paper(alg: str, n: int) -> float:
    return float(PAPER[alg]) * float(n) ** 3


def executed(alg: str, n: int) -> float:
    return float(EXECUTED[alg]) * float(n) ** 3


def nominal(n: int) -> float:
    return float(NOMINAL) * float(n) ** 3


def complex_gemm(n: int, three_mult: bool = True) -> float:
    """Real flops of one complex n x n product: 3 real GEMMs with Gauss's
    trick (Sec. 2, Proposition "matrix mult"), else 4."""
    return (6.0 if three_mult else 8.0) * float(n) ** 3
