"""Mixed-precision Frobenius inversion (FP32 start, Newton-Schulz refinement
with FP64-accurate residuals on the BF16 tensor cores) against the oracle.

The result must meet the FP64 targets: ||M X - I||_F/(||M||_F ||X||_F) <=
1e-13, and a forward error against the oracle's complex LU inverse within
32 n kappa(M) u64 plus kappa times the residual at which the refinement stops
(its tolerance is 1e-14).  The residual the refinement measured on the device
(info.residual, from the digit-split products) must agree with the residual
recomputed in FP64 on the host, to the resolution of both.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import metrics
from paper_2208_01239_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


def _refined_bound(m, x, ref):
    """Forward-error gate for a refined inverse X against the oracle's
    reference inverse: X - M^{-1} = M^{-1} (M X - I), so ||X - M^{-1}||_max <=
    ||M^{-1}||_2 ||M X - I||_F (in FP64 on the host), relative to
    ||M^{-1}||_max; plus the reference's own error, at most 16 kappa(M) u
    above its measured distance to LAPACK's inverse."""
    n = m.shape[0]
    minv = np.linalg.inv(m)
    scale = max(np.abs(minv.real).max(), np.abs(minv.imag).max())
    r = np.linalg.norm(m @ x - np.eye(n))
    return (np.linalg.norm(minv, 2) * r / scale + metrics.forward_error(ref, minv) +
            16 * np.linalg.cond(m) * U64)


@pytest.fixture(scope="module")
def F():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    return frob


def test_mixed_tf32_is_unsupported(F):
    """FROB_MIXED_TF32 has no path of its own: every entry point refuses it."""
    m = torch.from_numpy(W.gaussian(16, 1, seed=1)).cuda()
    for f in (F.frob_inv, F.frob_inv_hpd, F.cplx_lu_inv, F.cplx_chol_inv):
        with pytest.raises(F.FrobError) as e:
            f(m, prec="mixed_tf32")
        assert e.value.status == F.FROB_ERR_UNSUPPORTED


@pytest.mark.parametrize("route", ["frob_inv", "cplx_lu_inv"])
@pytest.mark.parametrize("n", [1, 7, 33, 64, 100, 128, 200, 256, 512])
def test_mixed_vs_oracle(F, route, n):
    """The mixed Frobenius form and its control (an FP32 complex-LU start with
    the same refinement) against the oracle, at the FP64 targets."""
    prec = "mixed_bf16"
    batch = 3 if n <= 256 else 2
    ms = W.gaussian(n, batch=batch, seed=7000 + n)
    r = getattr(F, route)(torch.from_numpy(ms).cuda(), prec=prec)
    x = r.x.cpu().numpy()
    info = r.info()
    for b in range(batch):
        ref = oracle.cplx_lu_inv(ms[b])
        res = metrics.residual_fro(ms[b], x[b])
        assert res <= 1e-13, res
        # refinement stops at the tolerance (1e-14): the forward error is
        # bounded by the attained residual (see _refined_bound)
        assert metrics.forward_error(x[b], ref) <= _refined_bound(ms[b], x[b], ref)
        # the device-side residual agrees with the host's FP64 evaluation to
        # the resolution of both: 7-digit products are within ~2^-46 of the
        # exact product relative to |M||X| (each operand truncated at 2^-50 of
        # a scale up to twice its row maximum, plus the dropped digit pairs),
        # and the host's own evaluation is noisy at ~sqrt(n) u
        tol = 0.05 * res + 2.0 ** -46 + 4 * np.sqrt(n) * U64
        assert abs(info["residual"][b] - res) <= tol, (info["residual"][b], res)
        assert info["ns_iters"][b] >= 1 or n == 1


def test_mixed_hpd_workload_kappa_1e4(F):
    """The HPD workload (kappa up to 1e4) through the general mixed route."""
    ms, qs, lams = W.hpd(256, batch=4, seed=21, return_parts=True)
    r = F.frob_inv(torch.from_numpy(ms).cuda(), prec="mixed_bf16")
    x = r.x.cpu().numpy()
    for b in range(4):
        exact = W.hpd_exact_inverse(qs[b], lams[b])
        kappa = lams[b].max() / lams[b].min()
        assert metrics.residual_fro(ms[b], x[b]) <= 1e-13
        assert metrics.forward_error(x[b], exact) <= 32 * 256 * kappa * U64


@pytest.mark.parametrize("route", ["frob_inv_hpd", "cplx_chol_inv"])
@pytest.mark.parametrize("n", [5, 64, 129, 512])
def test_mixed_hpd_route_vs_oracle(F, route, n):
    """frob_inv_hpd in the mixed precision: FP32 Cholesky-Frobenius start
    (Sec. 4.3), FP64-accurate refinement; and its control, an FP32 complex
    Cholesky start with the same refinement; lower triangle read."""
    batch = 3 if n < 512 else 8
    ms, qs, lams = W.hpd(n, batch=batch, seed=8000 + n, return_parts=True)
    bad = ms.copy()
    bad[:, np.triu_indices(n, 1)[0], np.triu_indices(n, 1)[1]] = 9.0 + 9.0j  # upper triangle ignored
    r = getattr(F, route)(torch.from_numpy(bad).cuda(), prec="mixed_bf16")
    x = r.x.cpu().numpy()
    for b in range(batch):
        exact = W.hpd_exact_inverse(qs[b], lams[b])
        kappa = lams[b].max() / lams[b].min()
        res = metrics.residual_fro(ms[b], x[b])
        assert res <= 1e-13
        ref = oracle.cplx_chol_inv(ms[b])
        assert metrics.forward_error(x[b], ref) <= _refined_bound(ms[b], x[b], ref)
        assert metrics.forward_error(x[b], exact) <= _refined_bound(ms[b], x[b], exact)


@pytest.mark.parametrize("route,n", [("frob_inv", 33), ("frob_inv", 200), ("frob_inv", 512),
                                     ("frob_inv_hpd", 129), ("frob_inv_hpd", 512), ("cplx_lu_inv", 200),
                                     ("cplx_chol_inv", 512)])
def test_mixed_fine_tolerance(F, route, n):
    """A tolerance below 1e-14 selects 8-digit residual products (pairs
    s + t <= 9): the refinement then reaches relative residuals near 1e-16,
    also for the HPD workload whose large diagonal sets the row scales."""
    batch = 2
    if route in ("frob_inv", "cplx_lu_inv"):
        ms = W.gaussian(n, batch=batch, seed=9100 + n)
    else:
        ms = W.hpd(n, batch=batch, seed=9200 + n)
    r = getattr(F, route)(torch.from_numpy(ms).cuda(), prec="mixed_bf16", ns_tol=1e-15)
    x = r.x.cpu().numpy()
    info = r.info()
    for b in range(batch):
        res = metrics.residual_fro(ms[b], x[b])
        assert info["residual"][b] <= 1e-15
        assert res <= 2e-15, res
        ref = oracle.cplx_lu_inv(ms[b])
        kappa = np.linalg.cond(ms[b])
        assert metrics.forward_error(x[b], ref) <= 32 * n * kappa * U64


def test_mixed_reports_failure_instead_of_wrong_result(F):
    """kappa(M) ~ 2e6 with S = (1 - s^2) I: the FP32 start cannot resolve S.
    Every matrix is either refined to the FP64 target or reported
    FROB_ERR_NOT_CONVERGED; none is returned as OK with a poor residual."""
    m, _ = W.ill_conditioned(64, seed=3)
    ms = np.stack([m, W.gaussian(64, 1, seed=5)[0]])
    r = F.frob_inv(torch.from_numpy(ms).cuda(), prec="mixed_bf16", check=False)
    x = r.x.cpu().numpy()
    info = r.info()
    for b in range(2):
        if info["status"][b] == F.FROB_OK:
            assert metrics.residual_fro(ms[b], x[b]) <= 1e-13
        else:
            assert info["status"][b] == F.FROB_ERR_NOT_CONVERGED
    assert info["status"][1] == F.FROB_OK


def test_mixed_rejects_large_n(F):
    m = torch.zeros((1, 520, 520), dtype=torch.complex128, device="cuda")
    with pytest.raises(F.FrobError) as e:
        F.frob_inv(m, prec="mixed_bf16", ws=torch.empty(1024, dtype=torch.uint8, device="cuda"))
    assert e.value.status in (F.FROB_ERR_UNSUPPORTED, F.FROB_ERR_WORKSPACE, F.FROB_ERR_ARG)
