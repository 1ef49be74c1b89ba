"""Batched inversion of matrices of different orders (frob_inv_batched),
each result against the oracle, plus CUDA-graph capture and the 1024-matrix
uneven workload (n uniform in [32, 512], A, B iid N(0, 1)) in the mixed
precision."""
import numpy as np
import pytest
import torch

import oracle
from oracle import metrics
from paper_2208_01239_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24, "mixed_bf16": 2.0 ** -53}
SIZES = [1, 5, 31, 32, 33, 64, 100, 129, 200, 257, 512, 7, 64]


@pytest.fixture(scope="module")
def F():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    return frob


def _check(ms, xs, prec, info, hpd=False):
    for k, (m, x) in enumerate(zip(ms, xs)):
        m64 = m.astype(np.complex128)
        x = x.cpu().numpy().astype(np.complex128)
        ref = oracle.cplx_chol_inv(m64) if hpd else oracle.cplx_lu_inv(m64)
        n = m.shape[0]
        kappa = np.linalg.cond(m64)
        res = metrics.residual_fro(m64, x)
        assert res <= (1e-5 if prec == "fp32" else 1e-13), (k, n, res)
        if prec.startswith("mixed"):
            # X - M^{-1} = M^{-1} (M X - I): bounded by the attained residual,
            # plus the reference's own error (its distance to LAPACK + 16 kappa u)
            minv = np.linalg.inv(m64)
            scale = max(np.abs(minv.real).max(), np.abs(minv.imag).max())
            bound = (np.linalg.norm(minv, 2) * np.linalg.norm(m64 @ x - np.eye(n)) / scale +
                     metrics.forward_error(ref, minv) + 16 * kappa * U[prec])
        else:
            bound = 32 * n * kappa * U[prec]
        assert metrics.forward_error(x, ref) <= bound, (k, n)
        assert info["status"][k] == 0


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed_bf16"])
@pytest.mark.parametrize("op", ["frob_inv", "cplx_lu_inv"])
def test_batched_uneven_vs_oracle(F, op, prec):
    # cplx_lu_inv with mixed_bf16 is the refined control (FP32 complex-LU start)
    dt = np.complex64 if prec == "fp32" else np.complex128
    ms = [W.gaussian(n, 1, seed=900 + i, dtype=dt)[0] for i, n in enumerate(SIZES)]
    xs, info = F.frob_inv_batched([torch.from_numpy(m).cuda() for m in ms], op=op, prec=prec)
    _check(ms, xs, prec, info)


@pytest.mark.parametrize("op", ["frob_inv_hpd", "cplx_chol_inv"])
def test_batched_uneven_hpd(F, op):
    ms = [W.hpd(n, 1, seed=950 + i)[0] for i, n in enumerate(SIZES)]
    xs, info = F.frob_inv_batched([torch.from_numpy(m).cuda() for m in ms], op=op, prec="fp64")
    _check(ms, xs, "fp64", info, hpd=True)


def test_batched_singular_member_reported(F):
    ms = [W.gaussian(n, 1, seed=i)[0] for i, n in enumerate([40, 70, 40])]
    ms[1][:, 3] = 0.0                                   # singular (zero column)
    xs, info = F.frob_inv_batched([torch.from_numpy(m).cuda() for m in ms], check=False)
    assert list(info["status"]) == [F.FROB_OK, F.FROB_ERR_SINGULAR, F.FROB_OK]


def test_batched_cuda_graph_capture_and_replay(F):
    ns = [33, 64, 100, 200, 64]
    plan = F.Batched(ns, op="frob_inv", prec="mixed_bf16")
    ms1 = [W.gaussian(n, 1, seed=70 + i)[0] for i, n in enumerate(ns)]
    for dst, m in zip(plan.inputs, ms1):
        dst.copy_(torch.from_numpy(m))
    plan.run()                                          # first call: sets kernel attributes
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    ms2 = [W.gaussian(n, 1, seed=80 + i)[0] for i, n in enumerate(ns)]
    for dst, m in zip(plan.inputs, ms2):
        dst.copy_(torch.from_numpy(m))
    g.replay()
    torch.cuda.synchronize()
    _check(ms2, plan.outputs, "mixed_bf16", plan.info())


def test_config4_uneven_1024_mixed(F):
    """1024 matrices, n ~ U{32..512}, A, B iid N(0,1): mixed precision with
    refinement; every result meets the FP64 residual target, eight sampled
    results agree with the oracle."""
    sizes, mats = W.uneven_batch(1024, 32, 512, seed=4)
    plan = F.Batched(sizes, op="frob_inv", prec="mixed_bf16")
    for dst, m in zip(plan.inputs, mats):
        dst.copy_(torch.from_numpy(m))
    plan.run()
    torch.cuda.synchronize()
    info = plan.info()
    assert (info["status"] == 0).all(), np.bincount(info["status"])
    assert info["residual"].max() <= 1e-13
    # residual of every result, recomputed in FP64 on the GPU by torch
    worst = 0.0
    for m, x in zip(mats, plan.outputs):
        md = torch.from_numpy(m).cuda()
        r = md @ x - torch.eye(m.shape[0], dtype=md.dtype, device="cuda")
        worst = max(worst, (torch.linalg.norm(r) / (torch.linalg.norm(md) * torch.linalg.norm(x))).item())
    assert worst <= 1e-13, worst
    g = np.random.default_rng(0)
    for k in g.choice(1024, 8, replace=False):
        m = mats[k]
        x = plan.outputs[k].cpu().numpy()
        kappa = np.linalg.cond(m)
        res = metrics.residual_fro(m, x)
        assert metrics.forward_error(x, oracle.cplx_lu_inv(m)) <= 32 * m.shape[0] * kappa * U["fp64"] + \
            4 * np.sqrt(m.shape[0]) * kappa * res


@pytest.mark.parametrize("part", ["B", "auto"])
def test_batched_part_options(F, part):
    """The part options through the uneven-order driver: the padding block
    is i I (B factored) or (1 + i) I (either part), so padded buckets stay
    invertible in the factored part; a matrix with a singular real part is
    inverted, every result against the oracle."""
    import numpy as np
    import torch
    import oracle
    from oracle import metrics
    g = np.random.default_rng(55)
    sizes = [37, 64, 5, 100]
    mats = [g.standard_normal((n, n)) + 1j * g.standard_normal((n, n)) for n in sizes]
    mats[0][:, 4] = mats[0][:, 4].imag * 1j  # real part of column 4 is zero: A singular
    outs, info = F.frob_inv_batched([torch.from_numpy(m).cuda() for m in mats], part=part)
    assert list(info["status"]) == [F.FROB_OK] * len(sizes)
    for m, x in zip(mats, outs):
        n = m.shape[0]
        assert metrics.forward_error(x.cpu().numpy(), oracle.cplx_lu_inv(m)) <= 32 * n * np.linalg.cond(m) * 2.0 ** -53
