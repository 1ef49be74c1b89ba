"""A batch of two or more matrices runs as two slices on two internal streams
(forked from the caller's stream and joined back).  Every matrix goes
through the same kernels and tile decompositions whatever the batch around
it, so the FP64 / FP32 results of a batched call must equal, bit for bit,
those of calls on each matrix alone; odd batches give slices of unequal size.
(The mixed precisions sum residual norms with atomics, whose order varies, so
they are checked against the FP64 targets elsewhere instead.)
"""
import numpy as np
import pytest
import torch

from paper_2208_01239_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    return frob


def _singles(fn, ms, prec):
    return np.stack([fn(torch.from_numpy(ms[b:b + 1]).cuda(), prec=prec).x.cpu().numpy()[0]
                     for b in range(ms.shape[0])])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("route,n,batch", [("frob_inv", 96, 3), ("frob_inv", 160, 2), ("frob_inv_hpd", 160, 5),
                                           ("cplx_lu_inv", 100, 3), ("cplx_chol_inv", 130, 3)])
def test_batched_equals_single_calls(F, prec, route, n, batch):
    if route in ("frob_inv_hpd", "cplx_chol_inv"):
        ms = W.hpd(n, batch, seed=900 + n)
    else:
        ms = W.gaussian(n, batch, seed=950 + n)
    if prec == "fp32":
        ms = ms.astype(np.complex64)
    fn = getattr(F, route)
    whole = fn(torch.from_numpy(ms).cuda(), prec=prec).x.cpu().numpy()
    alone = _singles(fn, ms, prec)
    assert np.array_equal(whole, alone)


def test_slice_info_offsets(F):
    """A failure in the second slice is reported at its own index."""
    n, batch = 64, 4
    ms = W.gaussian(n, batch, seed=77)
    ms[3][:, 5] = 0.0  # singular: column 5 of matrix 3 (in the second slice)
    r = F.frob_inv(torch.from_numpy(ms).cuda(), check=False)
    info = r.info()
    assert list(info["status"][:3]) == [F.FROB_OK] * 3
    assert info["status"][3] == F.FROB_ERR_SINGULAR


def test_autotuned_split_gives_the_same_results(F):
    """With the split autotuner on, the first call of a new shape runs the
    one- and two-slice forms and caches the faster; results are bit for bit
    those of the default split, and a graph capture does not tune."""
    ms = W.hpd(96, 6, seed=77)
    m = torch.from_numpy(ms).cuda()
    ref = F.frob_inv_hpd(m).x.cpu().numpy()
    F.autotune_clear()
    F.autotune(True)
    try:
        first = F.frob_inv_hpd(m).x.cpu().numpy()
        second = F.frob_inv_hpd(m).x.cpu().numpy()
        rep = F.autotune_report()
        key = (F.OP["frob_inv_hpd"], F.PREC["fp64"], 96, 6)
        assert key in rep and rep[key][0] in (1, 2) and rep[key][1] > 0 and rep[key][2] > 0
        assert np.array_equal(first, ref) and np.array_equal(second, ref)
        # a new shape under graph capture is not tuned
        m5 = torch.from_numpy(W.hpd(96, 5, seed=78)).cuda()
        out = torch.empty_like(m5)
        ws = torch.empty(F.workspace_bytes("frob_inv_hpd", 96, 5) + 256, dtype=torch.uint8, device="cuda")
        info = torch.zeros((5, 32), dtype=torch.uint8, device="cuda")
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            F.frob_inv_hpd(m5, out=out, ws=ws, info=info, check=False)  # eager first call: tunes this shape
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        F.autotune_clear()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            F.frob_inv_hpd(m5, out=out, ws=ws, info=info, check=False)
        assert F.autotune_report() == {}
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), F.frob_inv_hpd(m5).x.cpu().numpy())
    finally:
        F.autotune(False)
        F.autotune_clear()


def test_calls_from_short_lived_threads(F):
    """Each host thread's split streams are destroyed when it exits: batched
    calls from several short-lived threads, one after another and then
    concurrently, give the results of the calling thread."""
    import threading
    ms = W.gaussian(48, 2, seed=61)
    ref = F.frob_inv(torch.from_numpy(ms).cuda()).x.cpu().numpy()
    out = {}

    def work(k):
        torch.cuda.set_device(0)
        x = F.frob_inv(torch.from_numpy(ms).cuda()).x
        torch.cuda.synchronize()
        out[k] = x.cpu().numpy()

    for k in range(3):
        t = threading.Thread(target=work, args=(k,))
        t.start()
        t.join()
    ts = [threading.Thread(target=work, args=(10 + k,)) for k in range(3)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert sorted(out) == [0, 1, 2, 10, 11, 12]
    for v in out.values():
        assert np.array_equal(v, ref)
