"""Pins for the oracle's Newton drivers (Sec. 5.3-5.5 of Dai, Lim and Ye):
the matrix sign function, the Sylvester / Lyapunov equation through the sign
of a block matrix, and the polar decomposition.  Each is checked against a
result fixed by construction (the paper's "work backwards" generators: the
answer is known in closed form), against brute force (a Kronecker-product
linear system for Sylvester), and the stopping rule against the fixed-step
iteration."""
import numpy as np
import pytest

import oracle
from paper_2208_01239_gb300 import workloads as W


def _sign_case(n, seed):
    x, s = W.sign_case(n, seed=seed)
    return x, s


@pytest.mark.parametrize("n", [1, 2, 5, 12, 20])
def test_sign_closed_form(oracle_lib, n):
    x, s = _sign_case(n, 30 + n)
    got, steps = oracle.newton(x, 0, 1e-13, 100)
    assert 1 <= steps < 100
    assert np.abs(got - s).max() <= 1e-10 * np.abs(s).max()


def test_sign_scalar_is_sign_of_real_part(oracle_lib):
    for z, want in ((2.5 - 3j, 1.0), (-0.2 + 7j, -1.0), (1e-3 + 0j, 1.0)):
        got, _ = oracle.newton(np.array([[z]]), 0, 1e-15, 200)
        assert abs(got[0, 0] - want) < 1e-14


def test_stopping_rule_against_fixed_steps(oracle_lib):
    """The iterate returned after k steps is the fixed-step iterate X_k, bit
    for bit, and k is the first step whose relative change in the max norm is
    at most eps."""
    x, _ = _sign_case(16, 5)
    eps = 1e-3
    got, k = oracle.newton(x, 0, eps, 100)
    assert np.array_equal(got, oracle.sign_newton(x, k))
    rel = []
    for j in range(1, k + 1):
        a, b = oracle.sign_newton(x, j), oracle.sign_newton(x, j - 1)
        rel.append(np.abs(a - b).max() / np.abs(a).max())
    assert rel[-1] <= eps and all(r > eps for r in rel[:-1])


def test_zero_steps(oracle_lib):
    x, _ = _sign_case(6, 2)
    got, k = oracle.newton(x, 0, 1e-3, 0)
    assert k == 0 and np.array_equal(got, x)


@pytest.mark.parametrize("n", [1, 4, 15])
def test_polar_closed_form(oracle_lib, n):
    x, u, p = W.polar_case(n, seed=40 + n)
    q, pm, steps = oracle.polar(x, 1e-13, 100)
    assert 1 <= steps < 100
    assert np.abs(q - u).max() <= 1e-9
    assert np.abs(pm - p).max() <= 1e-9 * np.abs(p).max()
    assert np.abs(q.conj().T @ q - np.eye(n)).max() <= 1e-12      # unitary
    assert np.abs(pm - pm.conj().T).max() <= 1e-10 * np.abs(pm).max()  # Hermitian


@pytest.mark.parametrize("p,q,lyap", [(5, 7, False), (6, 6, True), (1, 3, False)])
def test_sylvester_closed_form(oracle_lib, p, q, lyap):
    a, b, c, y = W.sylvester_case(p, q, seed=50 + p + q, lyapunov=lyap)
    got, steps = oracle.sylvester(a, b, c, 1e-13, 100)
    assert 1 <= steps < 100
    assert np.abs(got - y).max() <= 1e-9 * np.abs(y).max()


def test_sylvester_against_kronecker_brute_force(oracle_lib):
    """A Y + Y B = C as (A (x) I_q + I_p (x) B^T) vec(Y) = vec(C), row-major
    vec, solved directly; A and B with spectra in the right half plane."""
    g = np.random.default_rng(12)
    p, q = 4, 5
    a = 0.3 * (g.standard_normal((p, p)) + 1j * g.standard_normal((p, p))) + 3 * np.eye(p)
    b = 0.3 * (g.standard_normal((q, q)) + 1j * g.standard_normal((q, q))) + 2 * np.eye(q)
    c = g.standard_normal((p, q)) + 1j * g.standard_normal((p, q))
    k = np.kron(a, np.eye(q)) + np.kron(np.eye(p), b.T)
    yref = np.linalg.solve(k, c.ravel()).reshape(p, q)
    got, _ = oracle.sylvester(a, b, c, 1e-14, 100)
    assert np.abs(got - yref).max() <= 1e-11 * np.abs(yref).max()
