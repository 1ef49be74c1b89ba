"""Differentiation through Frobenius inversion, on the GPU.

* The adjoint kernel (-X^H G X^H) against the oracle's plain-loop adjoint.
  Both are sums of products, so the bound is the usual GEMM one:
  |diff| <= 16 n u (|X|^T |G| |X|^T) elementwise (max norm).
* FrobInv's gradient against torch.linalg.inv's (a library route).
* The sign-iteration loss against directional central finite differences
  computed with the library's forward pass only, and its forward value
  against the oracle's sign iteration.
* Checkpointing gives the same gradient with a lower peak memory.
* The 16 x n = 1024 complex64 workload with 10 Newton steps.  There every
  eigenvalue of M = (A + iB), A, B ~ N(0,1)/sqrt(n) + 2I, lies in a disc of
  radius ~sqrt(2) about 2 + 2i, so sign(M) = I exactly and the gradient of
  Re tr(W^H sign(M)) is zero up to FP32 rounding; the non-degenerate case is
  covered by a shifted workload whose eigenvalues straddle the imaginary axis.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2208_01239_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U = {torch.complex128: 2.0 ** -53, torch.complex64: 2.0 ** -24}


@pytest.fixture(scope="module")
def A():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    from paper_2208_01239_gb300 import autograd
    return frob, autograd


def _rand(n, batch, seed, dtype=np.complex128):
    g = np.random.default_rng(seed)
    return (g.standard_normal((batch, n, n)) + 1j * g.standard_normal((batch, n, n))).astype(dtype)


@pytest.mark.parametrize("n", [1, 5, 64, 130])
@pytest.mark.parametrize("dtype", [torch.complex128, torch.complex64])
def test_adjoint_vs_oracle(A, n, dtype):
    frob, _ = A
    npdt = np.complex128 if dtype == torch.complex128 else np.complex64
    x = _rand(n, 2, 10 + n, npdt)
    g = _rand(n, 2, 20 + n, npdt)
    got = frob.inv_adjoint(torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda()).cpu().numpy()
    for b in range(2):
        x64, g64 = x[b].astype(np.complex128), g[b].astype(np.complex128)
        ref = oracle.inv_adjoint(x64, g64)
        bound = 16 * n * U[dtype] * (np.abs(x64).T @ np.abs(g64) @ np.abs(x64).T)
        assert np.all(np.abs(got[b] - ref) <= bound + 1e-300)


def test_autograd_matches_torch_linalg_inv(A):
    _, ag = A
    n = 40
    m0 = torch.from_numpy(_rand(n, 2, 1) + 3 * np.sqrt(n) * np.eye(n)).cuda()
    w = torch.from_numpy(_rand(n, 2, 2)).cuda()
    m1 = m0.clone().requires_grad_(True)
    (w.conj() * ag.frob_inverse(m1)).real.sum().backward()
    m2 = m0.clone().requires_grad_(True)
    (w.conj() * torch.linalg.inv(m2)).real.sum().backward()
    diff = (m1.grad - m2.grad).abs().max().item()
    assert diff <= 1e-12 * m2.grad.abs().max().item()


def _shifted(n, batch, seed, dtype=np.complex128):
    """A, B ~ N(0,1)/sqrt(n) plus +-2 on the diagonal (half each): eigenvalues
    on both sides of the imaginary axis."""
    g = np.random.default_rng(seed)
    d = np.where(np.arange(n) < n // 2, 2.0, -2.0)
    a = g.standard_normal((batch, n, n)) / np.sqrt(n) + np.diag(d)
    b = g.standard_normal((batch, n, n)) / np.sqrt(n) + np.diag(d)
    return (a + 1j * b).astype(dtype)


def test_sign_forward_vs_oracle(A):
    _, ag = A
    n = 48
    m = _shifted(n, 1, 3)
    s = ag.sign_newton(torch.from_numpy(m).cuda(), iters=6, checkpoint=False).cpu().numpy()[0]
    ref = oracle.sign_newton(m[0], 6)
    assert np.abs(s - ref).max() <= 1e-10 * np.abs(ref).max()


def test_sign_gradient_finite_difference(A):
    _, ag = A
    n, iters = 24, 3
    m0 = torch.from_numpy(_shifted(n, 1, 4)).cuda()
    w = torch.from_numpy(_rand(n, 1, 5)).cuda()
    d = torch.from_numpy(_rand(n, 1, 6)).cuda()
    m = m0.clone().requires_grad_(True)
    ag.sign_loss(m, w, iters).backward()
    an = (m.grad.conj() * d).real.sum().item()
    h = 1e-6
    with torch.no_grad():
        lp = ag.sign_loss(m0 + h * d, w, iters, checkpoint=False).item()
        lm = ag.sign_loss(m0 - h * d, w, iters, checkpoint=False).item()
    fd = (lp - lm) / (2 * h)
    assert abs(fd - an) <= 1e-6 * max(1.0, abs(an))


def test_checkpointing_same_gradient_less_memory(A):
    _, ag = A
    n, iters = 256, 6
    m0 = torch.from_numpy(_shifted(n, 2, 7)).cuda()
    w = torch.from_numpy(_rand(n, 2, 8)).cuda()
    grads, peaks = [], []
    for ck in (False, True):
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        base = torch.cuda.memory_allocated()
        m = m0.clone().requires_grad_(True)
        ag.sign_loss(m, w, iters, checkpoint=ck).backward()
        torch.cuda.synchronize()
        peaks.append(torch.cuda.max_memory_allocated() - base)
        grads.append(m.grad.clone())
    assert torch.allclose(grads[0], grads[1], rtol=0, atol=1e-12 * grads[0].abs().max().item())
    assert peaks[1] < peaks[0]


def test_config5_sign_batch16_n1024_fp32(A):
    """16 x n = 1024 complex64, A, B ~ N(0,1)/sqrt(n) + 2I, W Gaussian, 10
    Newton steps with checkpointing: sign(M) = I, gradient ~ 0, and the same
    as through torch.linalg.inv."""
    _, ag = A
    m_np, w_np = W.sign_workload(n=1024, batch=16, seed=5, w_seed=6)
    m0 = torch.from_numpy(m_np).cuda()
    w = torch.from_numpy(w_np).cuda()
    with torch.no_grad():
        s = ag.sign_newton(m0, 10, checkpoint=False)
    eye = torch.eye(1024, dtype=s.dtype, device=s.device)
    assert (s - eye).abs().max().item() <= 1e-4
    m = m0.clone().requires_grad_(True)
    loss = ag.sign_loss(m, w, 10, checkpoint=True)
    loss.backward()
    g = m.grad
    assert torch.isfinite(g.real).all() and torch.isfinite(g.imag).all()
    wmax = w.abs().max().item()
    assert g.abs().max().item() <= 1e-3 * wmax
    # torch.linalg.inv through the same iteration (reference route)
    m2 = m0.clone().requires_grad_(True)
    x = m2
    for _ in range(10):
        x = 0.5 * (x + torch.linalg.inv(x))
    (w.conj() * x).real.sum().backward()
    assert (g - m2.grad).abs().max().item() <= 1e-3 * wmax


def test_shifted_sign_gradient_fp32_vs_torch(A):
    """Non-degenerate sign gradient in complex64 against torch.linalg.inv."""
    _, ag = A
    n, iters = 256, 5
    m0 = torch.from_numpy(_shifted(n, 2, 9, np.complex64)).cuda()
    w = torch.from_numpy(_rand(n, 2, 10, np.complex64)).cuda()
    m = m0.clone().requires_grad_(True)
    ag.sign_loss(m, w, iters).backward()
    m2 = m0.clone().requires_grad_(True)
    x = m2
    for _ in range(iters):
        x = 0.5 * (x + torch.linalg.inv(x))
    (w.conj() * x).real.sum().backward()
    rel = ((m.grad - m2.grad).abs().max() / m2.grad.abs().max()).item()
    assert rel <= 1e-3, rel
