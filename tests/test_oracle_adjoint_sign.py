"""Pins for the oracle's adjoint and Newton sign iteration (no GPU).

* The adjoint -X^H G X^H is checked against central finite differences of
  the oracle's own complex LU inverse: for L(M) = Re <G, M^{-1}> (real inner
  product sum Re(conj(G) * Y)), the directional derivative along D equals
  Re <grad, D>.  Finite differences never use the adjoint formula.
* The sign iteration is checked against the closed form of Sec. 5.3:
  sign(Z J Z^{-1}) = Z diag(sign Re J) Z^{-1}.
"""
import numpy as np
import pytest

import oracle


def _rand(n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))


def _re_inner(a, b):
    return float(np.sum((np.conj(a) * b).real))


@pytest.mark.parametrize("n", [1, 3, 8, 20])
def test_adjoint_matches_finite_differences(oracle_lib, n):
    m = _rand(n, 10 + n) + 2 * n ** 0.5 * np.eye(n)
    g = _rand(n, 20 + n)
    d = _rand(n, 30 + n)
    x = oracle.cplx_lu_inv(m)
    grad = oracle.inv_adjoint(x, g)
    h = 1e-5
    lp = _re_inner(g, oracle.cplx_lu_inv(m + h * d))
    lm = _re_inner(g, oracle.cplx_lu_inv(m - h * d))
    fd = (lp - lm) / (2 * h)
    an = _re_inner(grad, d)
    assert abs(fd - an) <= 1e-7 * max(1.0, abs(an))


def test_adjoint_identity_pins():
    """X = I gives -G^... : -I^H G I^H = -G; a unitary X = U gives -U^H G U^H."""
    g = _rand(6, 1)
    np.testing.assert_allclose(oracle.inv_adjoint(np.eye(6), g), -g, rtol=0, atol=1e-15)
    u, _ = np.linalg.qr(_rand(6, 2))
    np.testing.assert_allclose(oracle.inv_adjoint(u, g), -(u.conj().T @ g @ u.conj().T), rtol=0, atol=1e-13)


@pytest.mark.parametrize("n", [4, 30])
def test_sign_newton_closed_form(oracle_lib, n):
    """X = Z J Z^{-1}, J diagonal with Re J of both signs (Sec. 5.3)."""
    g = np.random.default_rng(50 + n)
    p = n // 2
    re = np.concatenate([g.uniform(0.5, 2.0, p), -g.uniform(0.5, 2.0, n - p)])
    j = re + 1j * g.uniform(-1.0, 1.0, n)
    z = g.uniform(-1, 1, (n, n)) + 1j * g.uniform(-1, 1, (n, n)) + 3 * np.eye(n)
    x = z @ np.diag(j) @ np.linalg.inv(z)
    s = z @ np.diag(np.sign(re)).astype(complex) @ np.linalg.inv(z)
    got = oracle.sign_newton(x, 40)
    assert np.abs(got - s).max() <= 1e-9 * np.abs(s).max()
    # sign(X)^2 = I
    assert np.abs(got @ got - np.eye(n)).max() <= 1e-9


def test_sign_newton_zero_steps_is_identity_map():
    m = _rand(5, 3)
    np.testing.assert_array_equal(oracle.sign_newton(m, 0), m)
