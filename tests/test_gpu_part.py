"""The formula for invertible B (Sec. 4.2) and the automatic choice of the
factored real part, on the GPU against the oracle.

part="B": (A + iB)^{-1} = B^{-1}A(AB^{-1}A + B)^{-1} - i(AB^{-1}A + B)^{-1}.
part="auto": per matrix, A and B are both factored and the one whose U has
the larger min |u_kk| / max |u_kk| is used.  Bounds as in test_gpu_parity:
forward error <= 32 n kappa(M) u against the oracle's inverse, where the
factored part is well conditioned; where it is not, the error grows with its
condition number (reading 11), which the auto choice avoids."""
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


def _dev(m, prec="fp64"):
    return torch.from_numpy(np.ascontiguousarray(m)).to(torch.complex64 if prec == "fp32" else torch.complex128).cuda()


def _bound(m, prec):
    return 32 * m.shape[0] * np.linalg.cond(m) * U[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("n", [1, 33, 100, 257])
def test_part_b_general(F, prec, n):
    ms = W.gaussian(n, batch=2, seed=4000 + n)
    if prec == "fp32":
        ms = ms.astype(np.complex64)
    x = F.frob_inv(_dev(ms, prec), prec=prec, part="B").x.cpu().numpy().astype(np.complex128)
    for b in range(2):
        m64 = ms[b].astype(np.complex128)
        assert metrics.forward_error(x[b], oracle.frob_inv_b(m64)) <= _bound(m64, prec)
        assert metrics.residual_fro(m64, x[b]) <= (1e-13 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_singular_a_needs_b(F, prec):
    n = 80
    g = np.random.default_rng(41)
    a = g.standard_normal((n, n))
    a[:, 11] = 0.0
    m = a + 1j * g.standard_normal((n, n))
    ms = np.stack([W.gaussian(n, 1, seed=42)[0], m])
    if prec == "fp32":
        ms = ms.astype(np.complex64)
    ia = F.frob_inv(_dev(ms, prec), prec=prec, part="A", check=False).info()
    assert list(ia["status"]) == [F.FROB_OK, F.FROB_ERR_SINGULAR] and int(ia["bad_index"][1]) == 12
    for part in ("B", "auto"):
        r = F.frob_inv(_dev(ms, prec), prec=prec, part=part)
        x = r.x.cpu().numpy().astype(np.complex128)
        assert list(r.info()["status"]) == [F.FROB_OK, F.FROB_OK]
        for b in range(2):
            m64 = ms[b].astype(np.complex128)
            assert metrics.forward_error(x[b], oracle.cplx_lu_inv(m64)) <= _bound(m64, prec)


def test_auto_picks_the_better_conditioned_part(F):
    """Matrix 0: kappa(A) = 1e10, kappa(B) = 10; matrix 1 the other way round;
    matrix 2 both 10.  The A route loses ~kappa(A) u on matrix 0; auto keeps
    every matrix at the accuracy of the well-conditioned part, and on
    matrix 1 (A well conditioned, so A is chosen) it matches the A route bit
    for bit."""
    n = 96
    bad = W.kappa_controlled(n, 1e10, seed=51)
    good = W.kappa_controlled(n, 10.0, seed=52)
    ms = np.stack([bad.real + 1j * good.imag, good.real + 1j * bad.imag, good])
    xa = F.frob_inv(_dev(ms), part="A").x.cpu().numpy()
    xu = F.frob_inv(_dev(ms), part="auto").x.cpu().numpy()
    ref = [oracle.cplx_lu_inv(m) for m in ms]
    fe_a = [metrics.forward_error(xa[b], ref[b]) for b in range(3)]
    fe_u = [metrics.forward_error(xu[b], ref[b]) for b in range(3)]
    for b in range(3):
        assert fe_u[b] <= _bound(ms[b], "fp64") and fe_u[b] <= 1e-11
    assert fe_a[0] > 100 * fe_u[0]
    assert np.array_equal(xu[1], xa[1])


def test_auto_when_neither_part_is_invertible(F):
    """diag(1, i) (Sec. 4.2): A and B both singular, M invertible: auto
    reports the A factorization's failure (the almost sure variant is the
    route for such inputs)."""
    m = np.diag([1.0, 1j])
    info = F.frob_inv(_dev(m), part="auto", check=False).info()
    assert info["status"][0] == F.FROB_ERR_SINGULAR
    x = F.frob_inv(_dev(m), almost_sure=True, seed=3).x.cpu().numpy()
    assert np.abs(x - np.diag([1.0, -1j])).max() < 1e-14


def test_part_with_mixed_precision(F):
    n = 128
    g = np.random.default_rng(61)
    a = g.standard_normal((n, n))
    a[:, 5] = 0.0
    ms = np.stack([W.gaussian(n, 1, seed=62)[0], a + 1j * g.standard_normal((n, n))])
    for part in ("B", "auto"):
        r = F.frob_inv(_dev(ms), prec="mixed_bf16", part=part)
        x = r.x.cpu().numpy()
        for b in range(2):
            assert metrics.residual_fro(ms[b], x[b]) <= 1e-13
            assert metrics.forward_error(x[b], oracle.cplx_lu_inv(ms[b])) <= _bound(ms[b], "fp64")


def test_part_argument_errors(F):
    m = _dev(W.gaussian(8, 1, seed=1)[0])
    o = F._opts("fp64", part="B")
    o.part = 3
    with pytest.raises(F.FrobError) as e:
        F._call("frob_inv", m, "fp64", o, None, None, None, True)
    assert e.value.status == F.FROB_ERR_ARG
    with pytest.raises(F.FrobError) as e:
        F.frob_inv(m, almost_sure=True, part="B")
    assert e.value.status == F.FROB_ERR_ARG
    o = F._opts("fp64")
    o.fp64_gemm = 5
    with pytest.raises(F.FrobError) as e:
        F._call("frob_inv", m, "fp64", o, None, None, None, True)
    assert e.value.status == F.FROB_ERR_ARG


def test_auto_batched_equals_single_calls(F):
    """The choice is per matrix: a batch split over the two internal streams
    gives, bit for bit, the single-matrix results."""
    n = 70
    bad = W.kappa_controlled(n, 1e9, seed=71)
    good = W.kappa_controlled(n, 10.0, seed=72)
    ms = np.stack([bad.real + 1j * good.imag, good, good.real + 1j * bad.imag])
    whole = F.frob_inv(_dev(ms), part="auto").x.cpu().numpy()
    for b in range(3):
        alone = F.frob_inv(_dev(ms[b:b + 1]), part="auto").x.cpu().numpy()[0]
        assert np.array_equal(whole[b], alone)
