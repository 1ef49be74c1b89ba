"""Inversion over the iterated quadratic extension with m = 2 (Sec. 2.4,
Theorem "GFiter"): bicomplex matrices A + jB, j^2 = -1, j commuting with i.
The GPU route (Frobenius over C, complex inversions by frob_inv, complex
products by Gauss multiplication) against the oracle (the inverse of the
2n complex embedding [[A, -B], [B, A]]): forward error <= 32 (2n)
kappa(E) u with E the embedding, and the product identity."""
import numpy as np
import pytest
import torch

import oracle
from oracle import metrics

pytestmark = pytest.mark.gpu
U = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "mixed_bf16": 2.0 ** -53}


@pytest.fixture(scope="module")
def F():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    return frob


def _pair(n, batch, seed):
    g = np.random.default_rng(seed)
    a = g.standard_normal((batch, n, n)) + 1j * g.standard_normal((batch, n, n))
    b = g.standard_normal((batch, n, n)) + 1j * g.standard_normal((batch, n, n))
    return a, b


def _embed(a, b):
    return np.block([[a, -b], [b, a]])


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed_bf16"])
@pytest.mark.parametrize("n", [1, 7, 64, 130])
def test_bicomplex_vs_oracle(F, prec, n):
    a, b = _pair(n, 2, 900 + n)
    dt = torch.complex64 if prec == "fp32" else torch.complex128
    if prec == "fp32":
        a, b = a.astype(np.complex64), b.astype(np.complex64)
    y0, y1, _ = F.frob_inv_bicomplex(torch.from_numpy(a).to(dt).cuda(), torch.from_numpy(b).to(dt).cuda(), prec=prec)
    y0, y1 = y0.cpu().numpy().astype(np.complex128), y1.cpu().numpy().astype(np.complex128)
    for k in range(2):
        a64, b64 = a[k].astype(np.complex128), b[k].astype(np.complex128)
        r0, r1 = oracle.bicomplex_inv(a64, b64)
        e = _embed(a64, b64)
        bound = 32 * 2 * n * np.linalg.cond(e) * U[prec]
        got, ref = _embed(y0[k], y1[k]), _embed(r0, r1)
        assert metrics.forward_error(got, ref) <= bound
        p0 = a64 @ y0[k] - b64 @ y1[k]
        p1 = a64 @ y1[k] + b64 @ y0[k]
        tol = 1e-9 if prec != "fp32" else 1e-2
        assert np.abs(p0 - np.eye(n)).max() <= tol and np.abs(p1).max() <= tol


def test_bicomplex_failures(F):
    """Matrix 1: A singular (first inversion fails, its own index); matrix 2:
    A = I, B = iI makes X = 1 + ji a zero divisor ((1 + ji)(1 - ji) = 0): A
    is invertible but S = A + B A^{-1} B = 0, exactly in floating point
    here (every product is of 0, 1 and i), so the second inversion fails at
    its first step, reported as 2n + 1.  (With a random A and B = iA the
    rounding leaves S tiny but not zero, which is not a zero pivot.)"""
    n = 12
    a, b = _pair(n, 3, 95)
    a[1][:, 3] = 0.0
    a[2] = np.eye(n)
    b[2] = 1j * np.eye(n)
    y0, y1, info = F.frob_inv_bicomplex(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), check=False)
    inf = F.parse_info(info)
    assert list(inf["status"]) == [F.FROB_OK, F.FROB_ERR_SINGULAR, F.FROB_ERR_SINGULAR]
    assert 1 <= int(inf["bad_index"][1]) <= 2 * n
    assert int(inf["bad_index"][2]) == 2 * n + 1
    r0, r1 = oracle.bicomplex_inv(a[0], b[0])
    assert metrics.forward_error(_embed(y0.cpu().numpy()[0], y1.cpu().numpy()[0]), _embed(r0, r1)) <= 1e-11
