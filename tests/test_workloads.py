"""The seeded generators produce what their constructions promise (they
feed the closed-form pins and the benchmark): properties checked with
numpy, no GPU."""
import numpy as np
import pytest

from paper_2208_01239_gb300 import workloads as W


@pytest.mark.parametrize("n", [1, 6, 31])
def test_sign_case(n):
    x, s = W.sign_case(n, seed=100 + n)
    assert np.abs(s @ s - np.eye(n)).max() <= 1e-10 * max(1.0, np.abs(s).max() ** 2)
    assert np.abs(x @ s - s @ x).max() <= 1e-10 * np.abs(x).max() * np.abs(s).max() * n
    ev = np.linalg.eigvals(x)
    assert np.all(np.abs(ev.real) >= 0.5 - 1e-8)                  # kept away from the imaginary axis
    assert np.sum(ev.real > 0) == (n + 1) // 2


@pytest.mark.parametrize("n", [1, 8, 40])
def test_polar_case(n):
    x, u, p = W.polar_case(n, seed=200 + n)
    assert np.abs(u.conj().T @ u - np.eye(n)).max() <= 1e-13
    assert np.abs(p - p.conj().T).max() <= 1e-13 * np.abs(p).max()
    assert np.linalg.eigvalsh(0.5 * (p + p.conj().T)).min() > 0
    assert np.abs(x - u @ p).max() <= 1e-13 * np.abs(x).max()


@pytest.mark.parametrize("p,q,lyap", [(5, 7, False), (6, 6, True)])
def test_sylvester_case(p, q, lyap):
    a, b, c, y = W.sylvester_case(p, q, seed=300 + p + q, lyapunov=lyap)
    assert np.abs(a @ y + y @ b - c).max() <= 1e-12 * np.abs(c).max()
    for m in (a, b):
        ev = np.linalg.eigvals(m)
        assert np.all((ev.real > 9.0 - 1e-6) & (ev.real < 10.0 + 1e-6))
    if lyap:
        assert np.array_equal(b, a.conj().T)
    with pytest.raises(ValueError):
        W.sylvester_case(3, 4, lyapunov=True)


@pytest.mark.parametrize("n", [2, 16, 64])
def test_hpd_kappa(n):
    x = W.hpd_kappa(n, 10.0, seed=400 + n)
    assert np.array_equal(x, x.conj().T)
    lam = np.linalg.eigvalsh(x)
    assert lam.min() > 0
    assert abs(lam.max() / lam.min() - 10.0) <= 1e-9 * 10.0
