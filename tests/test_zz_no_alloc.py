"""frob_inv_hpd_noalloc: the HPD inversion for callers that cannot allocate
device memory (a framework plugin whose host owns every device buffer, a
latency-bound loop where a cudaMalloc could stall the device, a foreign
caller without a device allocator).  The library supplies the workspace from
a fixed scratch array; the caller passes only inputs, outputs and info.

The test calls the entry point through the C ABI twice in a row, on
different inputs, and checks each result two ways within the tolerance of
the parity tests: against frob_inv_hpd's (which uses a caller-provided
workspace), and against the closed-form inverse Q diag(1/lam) Q^H that the
generator M = Q diag(lam) Q^H fixes, which no GPU code computes.  It
builds and loads the library itself, so it passes alone in a fresh process as
well as after the other tests.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2208_01239_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def lib():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    L = frob.load()
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    L.frob_inv_hpd_noalloc.argtypes = [i32, i32, vp, i64, i64, vp, i64, i64, vp, vp]
    L.frob_inv_hpd_noalloc.restype = i32
    assert torch.cuda.is_available()
    return L, frob


def _fe(x, ref):
    d = x - ref
    num = max(np.abs(d.real).max(), np.abs(d.imag).max())
    den = max(np.abs(ref.real).max(), np.abs(ref.imag).max())
    return num / den


def _noalloc(L, m_dev):
    batch, n = m_dev.shape[0], m_dev.shape[-1]
    x = torch.empty_like(m_dev)
    info = torch.zeros((batch, 32), dtype=torch.uint8, device=m_dev.device)
    st = L.frob_inv_hpd_noalloc(n, batch, m_dev.data_ptr(), n, n * n, x.data_ptr(), n, n * n, info.data_ptr(),
                                torch.cuda.current_stream().cuda_stream)
    return st, x, info


def test_noalloc_matches_frob_inv_hpd_twice(lib):
    L, frob = lib
    n, batch = 256, 3
    for call, seed in enumerate((71, 72)):
        ms, qs, lams = W.hpd(n, batch=batch, seed=seed, return_parts=True)
        dm = torch.from_numpy(ms).cuda()
        st, x, info = _noalloc(L, dm)
        assert st == 0, f"call {call}: status {st}"
        torch.cuda.synchronize()
        frob.check_info(frob.parse_info(info), "frob_inv_hpd_noalloc")
        ref = frob.frob_inv_hpd(dm).x.cpu().numpy()
        got = x.cpu().numpy()
        for b in range(batch):
            kappa = lams[b].max() / lams[b].min()
            assert _fe(got[b], ref[b]) <= 32 * n * kappa * U64, f"call {call}, matrix {b}"
            exact = W.hpd_exact_inverse(qs[b], lams[b])
            assert _fe(got[b], exact) <= 32 * n * kappa * U64, f"call {call}, matrix {b} (closed form)"


def test_noalloc_rejects_problems_beyond_the_scratch(lib):
    L, _ = lib
    n = 2048  # needs 4 planes of 32 MiB
    dm = torch.zeros((1, n, n), dtype=torch.complex128, device="cuda")
    before = L.frob_kernel_launches()
    st, _, _ = _noalloc(L, dm)
    assert st == 7  # FROB_ERR_WORKSPACE, returned before any launch
    assert L.frob_kernel_launches() == before
