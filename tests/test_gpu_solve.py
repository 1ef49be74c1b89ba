"""Frobenius linear solve (Sec. 3) and the complex-LU solve baseline on the
GPU against the oracle's Frobenius solve and LAPACK (a library route).
Forward-error bound 32 n kappa(M) u, residual max|M X - B| small; the
ill-conditioned construction (A = I, B = Q N Q^T) against its closed form."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from oracle import metrics
from paper_2208_01239_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}


@pytest.fixture(scope="module")
def F():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    return frob


def _rand(shape, seed, dtype=np.complex128):
    g = np.random.default_rng(seed)
    return (g.standard_normal(shape) + 1j * g.standard_normal(shape)).astype(dtype)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n,nrhs", [(1, 1), (5, 2), (33, 1), (64, 3), (129, 1), (256, 8), (300, 65)])
def test_solve_vs_oracle(F, prec, n, nrhs):
    dt = np.complex64 if prec == "fp32" else np.complex128
    ms = _rand((2, n, n), 100 + n, dt)
    bs = _rand((2, n, nrhs), 200 + n, dt)
    for method in ("frob_solve", "cplx_lu_solve", "aug_real_solve"):
        x = getattr(F, method)(torch.from_numpy(ms).cuda(), torch.from_numpy(bs).cuda(), prec=prec).x.cpu().numpy()
        for b in range(2):
            m64, b64 = ms[b].astype(np.complex128), bs[b].astype(np.complex128)
            ref = oracle.frob_solve(m64, b64) if method == "frob_solve" else np.linalg.solve(m64, b64)
            kappa = np.linalg.cond(m64)
            assert metrics.forward_error(x[b], ref) <= 32 * n * kappa * U[prec], (method, b)


def test_solve_ill_conditioned_closed_form(F):
    """kappa(M) ~ 2e6 with kappa(A) = kappa(B) = 1: the case the paper singles
    out (Sec. 3, 5.2).  Forward error against x = (I - iB) b / (1 - s^2)."""
    m, minv = W.ill_conditioned(512, seed=3)
    b = _rand((512, 4), 5)
    xf = F.frob_solve(torch.from_numpy(m).cuda(), torch.from_numpy(b).cuda()).x.cpu().numpy()
    xl = F.cplx_lu_solve(torch.from_numpy(m).cuda(), torch.from_numpy(b).cuda()).x.cpu().numpy()
    xa = F.aug_real_solve(torch.from_numpy(m).cuda(), torch.from_numpy(b).cuda()).x.cpu().numpy()
    exact = minv @ b
    fe_f, fe_l = metrics.forward_error(xf, exact), metrics.forward_error(xl, exact)
    assert fe_f <= 1e-7, fe_f
    assert fe_l <= 1e-7, fe_l
    assert metrics.forward_error(xa, exact) <= 1e-7


def test_solve_singular_real_part_reported(F):
    m = np.diag([1.0, 1j])[None]
    with pytest.raises(F.FrobError) as e:
        F.frob_solve(torch.from_numpy(m).cuda(), torch.ones((1, 2, 1), dtype=torch.complex128, device="cuda"))
    assert e.value.status == F.FROB_ERR_SINGULAR


def test_aug_solve_singular_reported(F):
    """The augmented matrix of a singular M is singular (its determinant is
    |det M|^2): diag(0, 1, i) fails in the real LU of order 2n = 6."""
    m = np.stack([np.diag([0.0, 1.0, 1j]), np.diag([2.0, 1.0, 1j])])
    b = _rand((2, 3, 1), 9)
    r = F.aug_real_solve(torch.from_numpy(m).cuda(), torch.from_numpy(b).cuda(), check=False)
    info = r.info()
    assert list(info["status"]) == [F.FROB_ERR_SINGULAR, F.FROB_OK]
    assert 1 <= int(info["bad_index"][0]) <= 6
    assert metrics.forward_error(r.x.cpu().numpy()[1], np.linalg.solve(m[1], b[1])) <= 1e-15
