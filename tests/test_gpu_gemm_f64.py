"""The FP64 digit-product GEMM (frob_gemm_f64) against the exact product.

Reference values are exact: every product a_k b_k is split into two doubles
whose sum is exact (Veltkamp splitting and Dekker's product), and
math.fsum of those terms and the negated GPU result gives the GPU error
rounded once.  Two checks per sampled entry:

* the worst-case bound of the digit scheme, relative to the powers of two
  just above the row maximum of op(A) and the column maximum of op(B):
  |C - AB| <= K 2^-52 2^(e_i + f_j) + 2^-52 |C|  (digit truncation, dropped
  digit pairs and the fixed-point rounding together stay below K 2^-54);
* on Gaussian operands, the root-mean-square error is within 2x that of
  the correctly rounded product up to K ~ 1000 and 8x up to K = 16384 (the
  half-unit roundings of the chunks' low digit groups add up with K); FP64
  dot products give 10x to 100x, one digit fewer 50x or more.
"""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    return frob


def _split(x):
    c = 134217729.0 * x  # 2^27 + 1
    hi = c - (c - x)
    return hi, x - hi


def _two_prod(a, b):
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _exact_errors(opa, opb, c, idx, alpha=1.0, c0=None, beta=0.0):
    """fl(alpha op(A) op(B) + beta C0 - C) at the sampled (b, i, j), computed
    exactly and rounded once (alpha and beta powers of two)."""
    out = np.empty(len(idx))
    for n, (b, i, j) in enumerate(idx):
        p, e = _two_prod(opa[b, i, :], opb[b, :, j])
        terms = list(alpha * p) + list(alpha * e) + [-c[b, i, j]]
        if c0 is not None:
            terms.append(beta * c0[b, i, j])
        out[n] = math.fsum(terms)
    return out


def _exact_rounding_errors(opa, opb, idx):
    """fl(round(AB) - AB): the error of the correctly rounded product."""
    out = np.empty(len(idx))
    for n, (b, i, j) in enumerate(idx):
        p, e = _two_prod(opa[b, i, :], opb[b, :, j])
        terms = list(p) + list(e)
        r = math.fsum(terms)
        out[n] = math.fsum([r] + [-t for t in terms])
    return out


def _pow2_above(m):
    """Smallest power of two strictly above m (1 for m = 0)."""
    m = np.asarray(m, dtype=np.float64)
    e = np.where(m > 0, np.floor(np.log2(np.where(m > 0, m, 1.0))) + 1, 0.0)
    # floor(log2) can be off by one near powers of two
    e = np.where(np.ldexp(1.0, (e - 1).astype(np.int64)) > m, e - 1, e)
    e = np.where(np.ldexp(1.0, e.astype(np.int64)) <= m, e + 1, e)
    return np.ldexp(1.0, e.astype(np.int64))


def _samples(batch, M, N, count, seed):
    g = np.random.default_rng(seed)
    idx = [(int(g.integers(batch)), int(g.integers(M)), int(g.integers(N))) for _ in range(count)]
    # ragged tails and corners
    idx += [(batch - 1, M - 1, N - 1), (0, M - 1, 0), (0, 0, N - 1), (batch - 1, M // 2, N - 1)]
    return idx


def _operands(batch, M, N, K, ta, tb, seed, dist="gauss"):
    g = np.random.default_rng(seed)
    opa = g.standard_normal((batch, M, K))
    opb = g.standard_normal((batch, K, N))
    if dist == "spread":
        # rows and columns far apart in magnitude, entries within a row
        # spanning 2^+-20
        opa *= np.ldexp(1.0, g.integers(-300, 300, (batch, M, 1)))
        opb *= np.ldexp(1.0, g.integers(-300, 300, (batch, 1, N)))
        opa *= np.ldexp(1.0, g.integers(-20, 1, (batch, M, K)))
        opb *= np.ldexp(1.0, g.integers(-20, 1, (batch, K, N)))
    sa = np.ascontiguousarray(opa.transpose(0, 2, 1)) if ta else opa
    sb = np.ascontiguousarray(opb.transpose(0, 2, 1)) if tb else opb
    return opa, opb, sa, sb


def _bound(opa, opb, c, idx, K):
    out = np.empty(len(idx))
    for n, (b, i, j) in enumerate(idx):
        s = _pow2_above(np.max(np.abs(opa[b, i, :]))) * _pow2_above(np.max(np.abs(opb[b, :, j])))
        out[n] = K * 2.0 ** -52 * s + 2.0 ** -52 * abs(c[b, i, j])
    return out


SHAPES = [
    (256, 256, 256, 1, False, False),
    (300, 520, 777, 2, True, False),     # ragged tiles, two chunks, batch stride
    (520, 300, 1030, 1, False, True),
    (384, 640, 4100, 1, True, True),     # nine chunks, fixed-point unit 2^-49
    (1030, 1100, 256, 3, False, False),  # more tiles than SMs
    (256, 300, 16384, 1, False, True),   # 32 chunks
    # thin products (K <= 128: exponents and digits in one pass), as the
    # rank-32 updates of LU panels
    (2000, 480, 32, 1, False, False),
    (300, 129, 1, 2, True, True),
    (1030, 640, 100, 1, False, True),
    (384, 256, 200, 1, True, False),     # between: K padded to 256
]


@pytest.mark.parametrize("shape", SHAPES)
def test_gemm_f64_exact(F, shape):
    M, N, K, batch, ta, tb = shape
    opa, opb, sa, sb = _operands(batch, M, N, K, ta, tb, seed=M + 3 * N + 7 * K)
    c = F.gemm_f64(torch.from_numpy(sa).cuda(), torch.from_numpy(sb).cuda(), trans_a=ta, trans_b=tb).cpu().numpy()
    assert c.shape == (batch, M, N)
    assert np.all(np.isfinite(c))
    idx = _samples(batch, M, N, 160, seed=K)
    err = np.abs(_exact_errors(opa, opb, c, idx))
    bound = _bound(opa, opb, c, idx, K)
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"
    cr = _exact_rounding_errors(opa, opb, idx)
    rms, rms_cr = math.sqrt(np.mean(err ** 2)), math.sqrt(np.mean(cr ** 2))
    assert rms <= (2.0 if K <= 1100 else 8.0) * rms_cr, f"rms error {rms:.3g} vs correctly rounded {rms_cr:.3g}"
    # every entry against an FP64 product of the same operands: within the
    # FP64 product's own worst-case bound
    ref = opa @ opb
    lim = 2 * K * 2.0 ** -53 * (np.abs(opa) @ np.abs(opb)) + K * 2.0 ** -52 * (
        _pow2_above(np.max(np.abs(opa), axis=2))[:, :, None] * _pow2_above(np.max(np.abs(opb), axis=1))[:, None, :])
    assert np.all(np.abs(c - ref) <= lim)


def test_gemm_f64_scales(F):
    """Rows and columns 2^+-300 apart, entries within a row spanning 2^20:
    the error bound holds relative to each row's and column's own scale."""
    M, N, K, batch = 300, 260, 600, 2
    opa, opb, sa, sb = _operands(batch, M, N, K, False, False, seed=11, dist="spread")
    c = F.gemm_f64(torch.from_numpy(sa).cuda(), torch.from_numpy(sb).cuda()).cpu().numpy()
    idx = _samples(batch, M, N, 160, seed=5)
    err = np.abs(_exact_errors(opa, opb, c, idx))
    bound = _bound(opa, opb, c, idx, K)
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"


def test_gemm_f64_alpha_beta(F):
    M, N, K, batch = 260, 390, 520, 2
    opa, opb, sa, sb = _operands(batch, M, N, K, False, True, seed=21)
    c0 = np.random.default_rng(22).standard_normal((batch, M, N))
    out = torch.from_numpy(c0.copy()).cuda()
    r = F.gemm_f64(torch.from_numpy(sa).cuda(), torch.from_numpy(sb).cuda(), trans_b=True, alpha=2.0, beta=-0.5,
                   out=out)
    assert r is out
    c = out.cpu().numpy()
    idx = _samples(batch, M, N, 120, seed=23)
    err = np.abs(_exact_errors(opa, opb, c, idx, alpha=2.0, c0=c0, beta=-0.5))
    bound = np.array([2 * K * 2.0 ** -52 * _pow2_above(np.max(np.abs(opa[b, i]))) *
                      _pow2_above(np.max(np.abs(opb[b, :, j]))) + 2.0 ** -51 * (abs(c[b, i, j]) + abs(c0[b, i, j]))
                      for (b, i, j) in idx])
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"
    # beta = 0 never reads C: NaN there is overwritten
    out2 = torch.full((batch, M, N), float("nan"), dtype=torch.float64, device="cuda")
    F.gemm_f64(torch.from_numpy(sa).cuda(), torch.from_numpy(sb).cuda(), trans_b=True, beta=0.0, out=out2)
    assert torch.isfinite(out2).all()


def test_gemm_f64_zero_and_nonfinite(F):
    M, N, K = 300, 280, 400
    g = np.random.default_rng(31)
    a = g.standard_normal((1, M, K))
    b = g.standard_normal((1, K, N))
    a[0, 7, :] = 0.0        # zero row: exact zeros
    b[0, :, 9] = 0.0        # zero column
    a[0, 11, 5] = np.inf    # row 11 -> NaN
    b[0, 17, 13] = np.nan   # column 13 -> NaN
    c = F.gemm_f64(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()[0]
    assert np.all(c[7, :13] == 0.0) and np.all(c[7, 14:] == 0.0)
    assert np.all(c[:11, 9] == 0.0) and np.all(c[12:, 9] == 0.0)
    assert np.all(np.isnan(c[11, :])) and np.all(np.isnan(c[:, 13]))
    keep_r = np.ones(M, bool)
    keep_r[11] = False
    keep_c = np.ones(N, bool)
    keep_c[13] = False
    sub = c[keep_r][:, keep_c]
    assert np.all(np.isfinite(sub))
    with np.errstate(invalid="ignore"):  # the infinite row times zeros
        ref = (a[0] @ np.nan_to_num(b[0], nan=0.0))[keep_r][:, keep_c]
    scale = (_pow2_above(np.max(np.abs(a[0][keep_r]), axis=1))[:, None] *
             _pow2_above(np.max(np.abs(b[0][:, keep_c]), axis=0))[None, :])
    assert np.all(np.abs(sub - ref) <= 2 * K * 2.0 ** -52 * scale)


def test_gemm_f64_arguments(F):
    lib = F.load()
    x = torch.zeros((1, 256, 256), dtype=torch.float64, device="cuda")
    with pytest.raises(ValueError):
        F.gemm_f64(torch.zeros((1, 127, 256), dtype=torch.float64, device="cuda"), x)
    assert lib.frob_gemm_f64_workspace_bytes(256, 127, 256, 1) == 0
    assert lib.frob_gemm_f64_workspace_bytes(256, 256, 0, 1) == 0
    need = int(lib.frob_gemm_f64_workspace_bytes(256, 256, 256, 1))
    assert need >= 16 * 512 * 256
    ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    pad = (-ws.data_ptr()) % 256
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    c = torch.empty_like(x)
    st = torch.cuda.current_stream().cuda_stream
    args = (256, 256, 256, 1, x.data_ptr(), 256, 65536, 0, x.data_ptr(), 256, 65536, 0, c.data_ptr(), 256, 65536,
            1.0, 0.0)
    assert lib.frob_gemm_f64(*args, ws.data_ptr() + pad, need - 1, err.data_ptr(), st) == F.FROB_ERR_WORKSPACE
    assert lib.frob_gemm_f64(*args, ws.data_ptr() + pad + 8, need, err.data_ptr(), st) == F.FROB_ERR_WORKSPACE
    bad = list(args)
    bad[7] = 2  # transA neither 0 nor 1
    assert lib.frob_gemm_f64(*bad, ws.data_ptr() + pad, need, err.data_ptr(), st) == F.FROB_ERR_ARG
    bad = list(args)
    bad[5] = 255  # lda below K
    assert lib.frob_gemm_f64(*bad, ws.data_ptr() + pad, need, err.data_ptr(), st) == F.FROB_ERR_ARG
    assert lib.frob_gemm_f64(*args, ws.data_ptr() + pad, need, err.data_ptr(), st) == F.FROB_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0 and torch.all(c == 0)
