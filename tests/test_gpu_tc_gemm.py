"""The tcgen05 tensor-core GEMM against the exact product of its rounded
operands (FP64 on the host).

The operands are rounded to BF16 (round to nearest even) or TF32 (round to
nearest, ties away) exactly as the conversion kernel does, so the only error
left is the FP32 accumulation: |C - C_ref| <= 2 K 2^-24 (|A| |B|^T) + tiny.
"""
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


def round_bf16(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def round_tf32(x):
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x1000) & 0xFFFFE000
    return u.astype(np.uint32).view(np.float32)


@pytest.mark.parametrize("kind", ["bf16", "tf32"])
@pytest.mark.parametrize("shape", [(128, 128, 64, 1), (256, 384, 512, 2), (200, 130, 100, 3), (1, 1, 1, 1),
                                   (129, 257, 1000, 1), (512, 512, 512, 4),
                                   # more tiles than SMs: persistent CTAs take several tiles each and
                                   # reuse both TMEM accumulators
                                   (1100, 2300, 192, 2), (2048, 2048, 128, 3)])
def test_tc_gemm_exact_operands(F, kind, shape):
    M, N, K, batch = shape
    g = np.random.default_rng(M * 7 + N * 3 + K)
    a = g.standard_normal((batch, M, K)).astype(np.float32)
    b = g.standard_normal((batch, N, K)).astype(np.float32)
    c = F.gemm_tc(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), kind=kind).cpu().numpy()
    rnd = round_bf16 if kind == "bf16" else round_tf32
    ar, br = rnd(a).astype(np.float64), rnd(b).astype(np.float64)
    ref = ar @ br.transpose(0, 2, 1)
    bound = 2 * K * 2.0 ** -24 * (np.abs(ar) @ np.abs(br).transpose(0, 2, 1)) + 1e-30
    err = np.abs(c - ref)
    assert np.all(err <= bound), f"max err/bound {np.max(err / bound):.3g}"
