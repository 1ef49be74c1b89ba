"""The pins must catch plausible mistakes in the oracle.

``oracle.c`` compiled with ``-DORC_MUTANT=k`` plants one mistake (a wrong
operand order, a flipped sign, a dropped term, a missing conjugate, a
transposed operand, a wrong un-rotation sign, a wrong permutation order).  Each
planted copy must fail at least one of the checks below, which use the same
references as test_oracle_pins.py (closed forms, brute force, LAPACK on
unique results).  Mistakes are planted only in the CPU oracle.
"""
import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_2208_01239_gb300 import workloads as W

MUTANTS = {
    1: "X5 X2 instead of X2 X5 (Frobenius, explicit inverses)",
    2: "X3 + iX4 instead of X3 - iX4 (Frobenius with LU)",
    3: "X2 = B X1 instead of A + B X1 (Frobenius with LU)",
    4: "missing conjugate in complex Cholesky",
    5: "X1 X1^T instead of X1^T X1 (Frobenius with Cholesky)",
    6: "X3 + mu X4 instead of X3 - mu X4 (almost sure un-rotation)",
    7: "column swaps in forward order (left LU inverse)",
    8: "X^T instead of X^H in the adjoint",
    9: "X + X^{-1} instead of (X + X^{-1})/2 in the sign iteration",
    10: "y = y2 - y1 (the printed sign) in the Frobenius linear solve",
    11: "X^{-1} instead of X^{-H} in the polar iteration",
    12: "Y = +1/2 of the top-right block instead of -1/2 (Sylvester)",
    13: "P = Q X instead of Q^H X (polar decomposition)",
    14: "Y6 + i Y5 instead of Y6 - i Y5 (formula for invertible B)",
    15: "-Y1 read from the lower-left block (bicomplex inverse)",
}


def _pin_failures(o) -> list:
    fails = []
    g = np.random.default_rng(9)
    # brute force on small general matrices, every route
    for n in (2, 3, 4):
        m = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
        adj = o.adjugate_inv(m)
        routes = {
            "lu_left": lambda: o.cplx_lu_inv(m, left=True),
            "lu_right": lambda: o.cplx_lu_inv(m, left=False),
            "basic": lambda: o.frob_inv_basic(m),
            "lu": lambda: o.frob_inv_lu(m),
            "rand": lambda: o.frob_inv_rand(m, 0.37),
            "b": lambda: o.frob_inv_b(m),
        }
        for name, f in routes.items():
            try:
                if metrics.forward_error(f(), adj) > 1e-12:
                    fails.append(f"adjugate n={n} {name}")
            except oracle.OracleError:
                fails.append(f"adjugate n={n} {name} raised")
    # LAPACK on a larger general matrix (more pivoting)
    m = g.standard_normal((24, 24)) + 1j * g.standard_normal((24, 24))
    ref = np.linalg.inv(m)
    for left in (True, False):
        if metrics.forward_error(o.cplx_lu_inv(m, left=left), ref) > 1e-10:
            fails.append(f"lapack left={left}")
    # HPD closed form, both Cholesky routes
    ms, qs, lams = W.hpd(12, 1, seed=4, return_parts=True)
    exact = W.hpd_exact_inverse(qs[0], lams[0])
    for name, f in (("cplx_chol", o.cplx_chol_inv), ("frob_chol", o.frob_inv_chol)):
        try:
            if metrics.forward_error(f(ms[0]), exact) > 1e-9:
                fails.append(f"hpd {name}")
        except oracle.OracleError:
            fails.append(f"hpd {name} raised")
    # adjoint against central finite differences of the inverse
    n = 6
    m = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)) + 4 * np.eye(n)
    gg = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    d = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    h = 1e-5
    ip = lambda a, b: float(np.sum((np.conj(a) * b).real))
    fd = (ip(gg, o.cplx_lu_inv(m + h * d)) - ip(gg, o.cplx_lu_inv(m - h * d))) / (2 * h)
    an = ip(o.inv_adjoint(o.cplx_lu_inv(m), gg), d)
    if abs(fd - an) > 1e-7 * max(1.0, abs(an)):
        fails.append("adjoint finite differences")
    # sign iteration against sign(Z J Z^{-1}) = Z sign(Re J) Z^{-1}
    re = np.array([1.0, 1.5, -0.7, -2.0])
    j = re + 1j * np.array([0.3, -0.2, 0.5, 0.1])
    z = g.standard_normal((4, 4)) + 3 * np.eye(4)
    x = z @ np.diag(j) @ np.linalg.inv(z)
    sref = z @ np.diag(np.sign(re)) @ np.linalg.inv(z)
    if np.abs(o.sign_newton(x, 40) - sref).max() > 1e-9 * np.abs(sref).max():
        fails.append("sign closed form")
    # polar decomposition and Sylvester equation against their constructions
    x, u, p = W.polar_case(5, seed=41)
    qf, pf, _ = o.polar(x, 1e-13, 100)
    if np.abs(qf - u).max() > 1e-9 or np.abs(pf - p).max() > 1e-9 * np.abs(p).max():
        fails.append("polar closed form")
    a, b, c, y = W.sylvester_case(4, 3, seed=51)
    yf, _ = o.sylvester(a, b, c, 1e-13, 100)
    if np.abs(yf - y).max() > 1e-9 * np.abs(y).max():
        fails.append("sylvester closed form")
    # bicomplex inverse: scalar closed form (a - jb) / (a^2 + b^2)
    a1, b1 = 1.3 - 0.4j, 0.7 + 0.9j
    y0, y1 = o.bicomplex_inv(np.array([[a1]]), np.array([[b1]]))
    d = a1 * a1 + b1 * b1
    if abs(y0[0, 0] - a1 / d) > 1e-14 or abs(y1[0, 0] + b1 / d) > 1e-14:
        fails.append("bicomplex scalar")
    # Frobenius linear solve against LAPACK
    m = g.standard_normal((9, 9)) + 1j * g.standard_normal((9, 9))
    rhs = g.standard_normal((9, 2)) + 1j * g.standard_normal((9, 2))
    if metrics.forward_error(o.frob_solve(m, rhs), np.linalg.solve(m, rhs)) > 1e-10:
        fails.append("frob_solve lapack")
    return fails


def test_clean_oracle_passes_the_pins(oracle_lib):
    assert _pin_failures(oracle.load()) == []


@pytest.mark.parametrize("k", sorted(MUTANTS), ids=lambda k: f"mutant{k}")
def test_planted_mistake_is_caught(oracle_lib, k):
    o = oracle.load(mutant=k)
    fails = _pin_failures(o)
    assert fails, f"planted mistake not caught: {MUTANTS[k]}"
