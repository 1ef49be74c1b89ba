"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the inversion arithmetic: it only draws matrices
(and, where a construction fixes it, the exact inverse implied by that
construction).  Every generator uses ``numpy.random.Generator(PCG64(seed))``
and fills the real part before the imaginary part.

Workloads (sizes follow the paper's experiments and the accuracy targets):

* :func:`gaussian` -- A, B iid N(0, 1): general complex inversion, n = 256.
* :func:`hpd` -- M = Q diag(lam) Q^H, Q from QR of a complex Gaussian matrix,
  lam log-uniform on [1, 1e4]; exact inverse Q diag(1/lam) Q^H.  Batch 64 of
  n = 512 (the HPD experiment of Sec. 5.6 uses Hermitian positive definite
  inputs of this kind).
* :func:`ill_conditioned` -- A = I, B = Q blockdiag([[0, -s], [s, 0]]) Q^T with
  Q random orthogonal and s = 1 - 1e-6: kappa(A) = kappa(B) = 1 while
  kappa(M) ~ 2e6 (the construction of Sec. 3, Theorem "illcond").  Since
  B^2 = -s^2 I, S = (1 - s^2) I and M^{-1} = (I - iB) / (1 - s^2).
* :func:`uneven_batch` -- n uniform in [32, 512], A, B iid N(0, 1).
* :func:`sign_workload` -- A, B iid N(0, 1)/sqrt(n) + 2I and a Gaussian W.
* :func:`kappa_controlled` -- the accuracy generator of Sec. 5.1:
  A = Q Lam Q^T / ||Lam||_F with kappa(A) = kappa, and B likewise.
* :func:`uniform01` -- A, B uniform on [0, 1] (the speed generator of Sec. 5.1).
* :func:`hpd_kappa` -- the HPD accuracy generator of Sec. 5.6:
  X = Q Lam Q^H / ||Lam||_F, Q from the QR factorization of a complex matrix
  uniform on [-1, 1] (real and imaginary parts), lam_1 = kappa, lam_n = 1,
  the rest uniform on [1, kappa].
* :func:`sign_case`, :func:`polar_case`, :func:`sylvester_case` -- the
  "work backwards" generators of Sec. 5.3-5.5, whose answers are known by
  construction: X = Z J Z^{-1} with sign(X) = Z sign(Re J) Z^{-1}; X = U P
  with U from the QR factorization of a random matrix and P = Z^H Z; and
  A = Z_A J_A Z_A^{-1}, B likewise (or B = A^H), C = A Y + Y B.  Entries of
  Z, Y are uniform on [-1, 1] in real and imaginary part, as in the paper.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def gaussian(n: int, batch: int = 1, seed: int = 1, dtype=np.complex128) -> np.ndarray:
    """(batch, n, n) complex matrices with A, B iid N(0, 1)."""
    g = _rng(seed)
    a = g.standard_normal((batch, n, n))
    b = g.standard_normal((batch, n, n))
    return (a + 1j * b).astype(dtype)


def uniform01(n: int, batch: int = 1, seed: int = 11, dtype=np.complex128) -> np.ndarray:
    g = _rng(seed)
    a = g.random((batch, n, n))
    b = g.random((batch, n, n))
    return (a + 1j * b).astype(dtype)


def _haar_unitary(g: np.random.Generator, n: int, complex_: bool) -> np.ndarray:
    """Q from the QR factorisation of a Gaussian matrix, with the phases of
    diag(R) folded in so that Q is Haar distributed."""
    if complex_:
        z = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    else:
        z = g.standard_normal((n, n))
    q, r = np.linalg.qr(z)
    d = np.diagonal(r)
    ph = d / np.abs(d)
    return q * ph[None, :]


def hpd(n: int, batch: int = 1, seed: int = 2, lam_lo: float = 1.0, lam_hi: float = 1e4,
        return_parts: bool = False):
    """Hermitian positive definite matrices M = Q diag(lam) Q^H.

    lam = 10**U(log10 lam_lo, log10 lam_hi).  The result is symmetrised as
    (M + M^H)/2.  With ``return_parts`` also returns (Q, lam) per matrix, from
    which the exact inverse Q diag(1/lam) Q^H follows."""
    g = _rng(seed)
    ms = np.empty((batch, n, n), dtype=np.complex128)
    qs, lams = [], []
    for t in range(batch):
        q = _haar_unitary(g, n, True)
        lam = 10.0 ** g.uniform(np.log10(lam_lo), np.log10(lam_hi), n)
        m = (q * lam[None, :]) @ q.conj().T
        ms[t] = 0.5 * (m + m.conj().T)
        qs.append(q)
        lams.append(lam)
    if return_parts:
        return ms, qs, lams
    return ms


def hpd_exact_inverse(q: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Q diag(1/lam) Q^H: the inverse fixed by the construction of :func:`hpd`."""
    return (q / lam[None, :]) @ q.conj().T


def ill_conditioned(n: int, seed: int = 3, s: float = 1.0 - 1e-6, dtype=np.complex128):
    """A = I, B = Q N Q^T, N = blockdiag([[0, -s], [s, 0]]), Q Haar orthogonal.

    Returns (M, Minv_exact) with Minv_exact = (I - iB)/(1 - s^2) evaluated from
    the rounded B (exact up to ||B^2 + s^2 I|| / (1 - s^2))."""
    if n % 2:
        raise ValueError("n must be even")
    g = _rng(seed)
    q = _haar_unitary(g, n, False)
    qn = np.empty_like(q)
    # (Q N)[:, 2i] = s Q[:, 2i+1], (Q N)[:, 2i+1] = -s Q[:, 2i]
    qn[:, 0::2] = s * q[:, 1::2]
    qn[:, 1::2] = -s * q[:, 0::2]
    b = qn @ q.T
    b = 0.5 * (b - b.T)
    m = (np.eye(n) + 1j * b).astype(dtype)
    minv = (np.eye(n) - 1j * b) / (1.0 - s * s)
    return m, minv


def uneven_sizes(count: int = 1024, n_lo: int = 32, n_hi: int = 512, seed: int = 4) -> np.ndarray:
    return _rng(seed).integers(n_lo, n_hi + 1, size=count)


def uneven_batch(count: int = 1024, n_lo: int = 32, n_hi: int = 512, seed: int = 4):
    """List of ``count`` Gaussian complex matrices with n ~ U{n_lo..n_hi}."""
    sizes = uneven_sizes(count, n_lo, n_hi, seed)
    g = _rng(seed + 1000)
    out = []
    for n in sizes:
        a = g.standard_normal((n, n))
        b = g.standard_normal((n, n))
        out.append(a + 1j * b)
    return sizes, out


def sign_workload(n: int = 1024, batch: int = 16, seed: int = 5, w_seed: int = 6, shift: float = 2.0,
                  dtype=np.complex64):
    """M = (A + iB) with A, B iid N(0,1)/sqrt(n) + shift*I, and a Gaussian W."""
    g = _rng(seed)
    a = g.standard_normal((batch, n, n)) / np.sqrt(n) + shift * np.eye(n)
    b = g.standard_normal((batch, n, n)) / np.sqrt(n) + shift * np.eye(n)
    gw = _rng(w_seed)
    w = gw.standard_normal((batch, n, n)) + 1j * gw.standard_normal((batch, n, n))
    return (a + 1j * b).astype(dtype), w.astype(dtype)


def kappa_controlled(n: int, kappa: float = 10.0, seed: int = 7) -> np.ndarray:
    """The accuracy generator of Sec. 5.1: Q from QR of a matrix uniform on
    [-1, 1]; Lam with lam_1 = +-kappa, lam_n = +-1 (random signs) and the rest
    uniform on [-kappa, -1] U [1, kappa]; A = Q Lam Q^T / ||Lam||_F; B alike."""
    g = _rng(seed)
    parts = []
    for _ in range(2):
        q, _r = np.linalg.qr(g.uniform(-1.0, 1.0, (n, n)))
        mag = np.empty(n)
        mag[0] = kappa
        if n > 1:
            mag[-1] = 1.0
        if n > 2:
            mag[1:-1] = g.uniform(1.0, kappa, n - 2)
        lam = mag * g.choice([-1.0, 1.0], n)
        parts.append((q * lam[None, :]) @ q.T / np.linalg.norm(lam))
    return parts[0] + 1j * parts[1]


def ulp_params() -> dict:
    """Unit roundoffs used by the tolerance derivations."""
    return {"f64": 2.0 ** -53, "f32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


def _unif_c(g: np.random.Generator, shape) -> np.ndarray:
    re = g.uniform(-1.0, 1.0, shape)
    im = g.uniform(-1.0, 1.0, shape)
    return re + 1j * im


def sign_case(n: int, seed: int = 21, re_lo: float = 0.5, re_hi: float = 1.5):
    """X = Z J Z^{-1} and its sign Z diag(sign(Re J)) Z^{-1} (Sec. 5.3).

    J is diagonal; its first ceil(n/2) entries have real part in [re_lo,
    re_hi] and the rest in [-re_hi, -re_lo] (kept away from zero), imaginary
    parts uniform on [-1, 1]; Z has real and imaginary parts uniform on
    [-1, 1].  Returns (X, sign(X)), complex128."""
    g = _rng(seed)
    z = _unif_c(g, (n, n))
    p = (n + 1) // 2
    mag = g.uniform(re_lo, re_hi, n)
    sgn = np.where(np.arange(n) < p, 1.0, -1.0)
    j = sgn * mag + 1j * g.uniform(-1.0, 1.0, n)
    zi = np.linalg.inv(z)
    return (z * j) @ zi, (z * sgn) @ zi


def polar_case(n: int, seed: int = 22):
    """X = U P with U unitary (from the QR factorization of a matrix with
    entries uniform on [-1, 1] in real and imaginary part) and P = Z^H Z for
    a second such matrix Z (Sec. 5.5).  Returns (X, U, P), complex128."""
    g = _rng(seed)
    y = _unif_c(g, (n, n))
    z = _unif_c(g, (n, n))
    u, _ = np.linalg.qr(y)
    p = z.conj().T @ z
    return u @ p, u, p


def sylvester_case(p: int, q: int, seed: int = 23, lyapunov: bool = False, re_lo: float = 9.0, re_hi: float = 10.0):
    """A Y + Y B = C with known Y (Sec. 5.4): A = Z_A J_A Z_A^{-1} with J_A
    diagonal, real parts uniform on [re_lo, re_hi] (so sign(A) = I) and
    imaginary parts uniform on [-1, 1]; B the same way with its own Z_B and
    J_B (or B = A^H when ``lyapunov``, which needs p == q); Y with entries
    uniform on [-1, 1] in real and imaginary part; C = A Y + Y B.  Returns
    (A, B, C, Y), complex128."""
    g = _rng(seed)

    def stable(k):
        z = _unif_c(g, (k, k))
        j = g.uniform(re_lo, re_hi, k) + 1j * g.uniform(-1.0, 1.0, k)
        return (z * j) @ np.linalg.inv(z)

    a = stable(p)
    if lyapunov:
        if p != q:
            raise ValueError("the Lyapunov equation has p == q")
        b = a.conj().T
    else:
        b = stable(q)
    y = _unif_c(g, (p, q))
    c = a @ y + y @ b
    return a, b, c, y


def hpd_kappa(n: int, kappa: float = 10.0, seed: int = 24) -> np.ndarray:
    """Hermitian positive definite X with kappa(X) = kappa (Sec. 5.6):
    Q from QR of a matrix with real and imaginary parts uniform on [-1, 1],
    Lam = diag(kappa, lam_2, ..., lam_{n-1}, 1) with the middle entries
    uniform on [1, kappa]; X = Q Lam Q^H / ||Lam||_F, symmetrised."""
    g = _rng(seed)
    q, _ = np.linalg.qr(_unif_c(g, (n, n)))
    lam = np.empty(n)
    lam[0] = kappa
    if n > 1:
        lam[-1] = 1.0
    if n > 2:
        lam[1:-1] = g.uniform(1.0, kappa, n - 2)
    x = (q * lam) @ q.conj().T / np.linalg.norm(lam)
    return 0.5 * (x + x.conj().T)
