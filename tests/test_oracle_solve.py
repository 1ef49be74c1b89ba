"""Pins for the oracle's Frobenius linear solve (Sec. 3, Algorithm "Linear
system with Frobenius inversion"): LAPACK's solve on general systems, the
closed form x = (I - iB) b / (1 - s^2) for the ill-conditioned construction,
and the 2 x 2 closed form."""
import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_2208_01239_gb300 import workloads as W


def _rand(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


@pytest.mark.parametrize("n,nrhs", [(1, 1), (5, 1), (33, 3), (64, 8)])
def test_frob_solve_vs_lapack(oracle_lib, n, nrhs):
    m = _rand((n, n), n)
    b = _rand((n, nrhs), n + 1)
    x = oracle.frob_solve(m, b)
    ref = np.linalg.solve(m, b)
    assert metrics.forward_error(x, ref) <= 64 * n * np.linalg.cond(m) * 2.0 ** -53 * 100
    assert np.abs(m @ x - b).max() <= 1e-10 * np.abs(m).max() * np.abs(x).max() * n


def test_frob_solve_vector_rhs(oracle_lib):
    m = _rand((12, 12), 3)
    b = _rand((12,), 4)
    np.testing.assert_allclose(oracle.frob_solve(m, b), np.linalg.solve(m, b), rtol=0, atol=1e-12)


def test_frob_solve_ill_conditioned_closed_form(oracle_lib):
    """A = I, B = Q N Q^T: M^{-1} = (I - iB)/(1 - s^2) (Sec. 3)."""
    m, minv = W.ill_conditioned(64, seed=9)
    b = _rand((64, 2), 10)
    assert metrics.forward_error(oracle.frob_solve(m, b), minv @ b) <= 1e-8


def test_frob_solve_2x2(oracle_lib):
    m = _rand((2, 2), 11)
    b = _rand((2,), 12)
    a_, b_, c_, d_ = m[0, 0], m[0, 1], m[1, 0], m[1, 1]
    inv = np.array([[d_, -b_], [-c_, a_]]) / (a_ * d_ - b_ * c_)
    assert metrics.forward_error(oracle.frob_solve(m, b), inv @ b) <= 1e-14


def test_frob_solve_singular_real_part_reported(oracle_lib):
    m = np.diag([1.0, 1j])
    with pytest.raises(oracle.OracleError):
        oracle.frob_solve(m, np.ones(2))
