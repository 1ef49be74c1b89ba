"""Newton drivers on the GPU (Sec. 5.3-5.5): matrix sign, polar
decomposition, Sylvester / Lyapunov equations, every step a Frobenius
inversion (or the complex-LU baseline route), against the oracle's drivers
and against the answers fixed by the paper's "work backwards" constructions.

Tolerances: the iterations converge quadratically to a limit fixed by the
construction, so once the relative change is below eps = 1e-10 the FP64
results agree with the closed form to ~kappa(Z)^2 u (asserted at 1e-9
relative, Z of order <= 257 with entries uniform on [-1, 1]); FP32 at 2e-3.
A smaller eps would sit at the rounding floor of the step (the relative
change of a converged iterate is ~kappa u, larger for the Frobenius inverse
than for LU), where the step count is decided by rounding noise.  At the paper's eps (1e-3 for sign and
polar) the GPU takes exactly the oracle's number of steps on these inputs
and its iterate matches the oracle's at that step to 1e-9."""
import numpy as np
import pytest
import torch

import oracle
from paper_2208_01239_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    from paper_2208_01239_gb300 import build, frob
    build.build()
    frob.load()
    return frob


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("route", ["frob", "cplx_lu"])
@pytest.mark.parametrize("n", [1, 33, 100, 257])
def test_sign_closed_form_fp64(F, route, n):
    x, s = W.sign_case(n, seed=300 + n)
    r = F.sign(torch.from_numpy(x).cuda(), route=route, eps=1e-10, kmax=100)
    got = r.out.cpu().numpy()
    _, k_or = oracle.newton(x, 0, 1e-10, 100)
    assert _rel(got, s) <= 1e-9
    assert abs(int(r.steps()[0]) - k_or) <= 1


@pytest.mark.parametrize("n", [16, 64])
def test_sign_paper_eps_matches_oracle_steps(F, n):
    x, _ = W.sign_case(n, seed=310 + n)
    r = F.sign(torch.from_numpy(x).cuda(), eps=1e-3, kmax=100)
    want, k = oracle.newton(x, 0, 1e-3, 100)
    assert int(r.steps()[0]) == k
    assert _rel(r.out.cpu().numpy(), want) <= 1e-9


def test_sign_batched_uneven_convergence(F):
    """A batch whose matrices stop after different numbers of steps: each
    result equals the single-matrix call's, bit for bit, and the step counts
    are the single calls' counts."""
    xs = np.stack([W.sign_case(48, seed=320 + b, re_lo=0.05 + 0.4 * b, re_hi=0.5 + 0.6 * b)[0] for b in range(3)])
    r = F.sign(torch.from_numpy(xs).cuda(), eps=1e-10, kmax=60)
    got, steps = r.out.cpu().numpy(), r.steps()
    for b in range(3):
        rb = F.sign(torch.from_numpy(xs[b]).cuda(), eps=1e-10, kmax=60)
        assert int(rb.steps()[0]) == int(steps[b])
        assert np.array_equal(rb.out.cpu().numpy(), got[b])
    assert len(set(steps.tolist())) > 1


def test_sign_fp32_and_mixed(F):
    x, s = W.sign_case(96, seed=330)
    r32 = F.sign(torch.from_numpy(x.astype(np.complex64)).cuda(), prec="fp32", eps=1e-4, kmax=100)
    assert _rel(r32.out.cpu().numpy().astype(np.complex128), s) <= 2e-3
    rm = F.sign(torch.from_numpy(x).cuda(), prec="mixed_bf16", eps=1e-10, kmax=100)
    assert _rel(rm.out.cpu().numpy(), s) <= 1e-9


@pytest.mark.parametrize("route", ["frob", "cplx_lu"])
@pytest.mark.parametrize("n", [1, 40, 97])
def test_polar_closed_form(F, route, n):
    xs, us, ps = zip(*[W.polar_case(n, seed=340 + n + b) for b in range(2)])
    r = F.polar(torch.from_numpy(np.stack(xs)).cuda(), route=route, eps=1e-10, kmax=100)
    q, p = (t.cpu().numpy() for t in r.out)
    for b in range(2):
        assert np.abs(q[b] - us[b]).max() <= 1e-9
        assert _rel(p[b], ps[b]) <= 1e-9
    qo, po, ko = oracle.polar(xs[0], 1e-10, 100)
    assert abs(int(r.steps()[0]) - ko) <= 1
    assert np.abs(q[0] - qo).max() <= 1e-9


@pytest.mark.parametrize("p,q,lyap", [(30, 50, False), (40, 40, True), (1, 7, False)])
def test_sylvester_closed_form(F, p, q, lyap):
    cases = [W.sylvester_case(p, q, seed=360 + p + q + b, lyapunov=lyap) for b in range(2)]
    a, b_, c, y = (np.stack(t) for t in zip(*cases))
    r = F.sylvester(torch.from_numpy(a).cuda(), None if lyap else torch.from_numpy(b_).cuda(),
                    torch.from_numpy(c).cuda(), eps=1e-10, kmax=100, lyapunov=lyap)
    got = r.out.cpu().numpy()
    for k in range(2):
        assert _rel(got[k], y[k]) <= 1e-9
    yo, ko = oracle.sylvester(a[0], b_[0], c[0], 1e-10, 100)
    assert np.abs(got[0] - yo).max() <= 1e-9 * np.abs(yo).max()
    assert abs(int(r.steps()[0]) - ko) <= 1


def test_sylvester_paper_eps(F):
    """The paper's tolerance for Sylvester (eps = 1e-1): the answer at the
    oracle's step count matches the oracle's."""
    a, b, c, y = W.sylvester_case(20, 12, seed=370)
    r = F.sylvester(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), torch.from_numpy(c).cuda(), eps=1e-1)
    yo, ko = oracle.sylvester(a, b, c, 1e-1, 100)
    assert int(r.steps()[0]) == ko
    assert np.abs(r.out.cpu().numpy() - yo).max() <= 1e-9 * np.abs(yo).max()


def test_zero_steps_and_singular(F):
    x, _ = W.sign_case(20, seed=380)
    r0 = F.sign(torch.from_numpy(x).cuda(), kmax=0)
    assert np.array_equal(r0.out.cpu().numpy(), x) and int(r0.steps()[0]) == 0
    xs = np.stack([x, np.zeros_like(x), x])
    r = F.sign(torch.from_numpy(xs).cuda(), eps=1e-10, check=False)
    info = r.info()
    assert list(info["status"]) == [F.FROB_OK, F.FROB_ERR_SINGULAR, F.FROB_OK]
    assert int(r.steps()[1]) == 0
    assert np.array_equal(r.out.cpu().numpy()[1], xs[1])
    good = F.sign(torch.from_numpy(x).cuda(), eps=1e-10).out.cpu().numpy()
    assert np.array_equal(r.out.cpu().numpy()[0], good)


def test_polar_and_sylvester_fp32(F):
    x, u, p = W.polar_case(40, seed=390)
    r = F.polar(torch.from_numpy(x.astype(np.complex64)).cuda(), prec="fp32", eps=1e-4)
    q, pm = (t.cpu().numpy().astype(np.complex128) for t in r.out)
    assert np.abs(q - u).max() <= 1e-3 and _rel(pm, p) <= 1e-3
    a, b, c, y = W.sylvester_case(20, 12, seed=391)
    ry = F.sylvester(*(torch.from_numpy(t.astype(np.complex64)).cuda() for t in (a, b, c)), prec="fp32", eps=1e-4)
    assert _rel(ry.out.cpu().numpy().astype(np.complex128), y) <= 1e-3


def test_sign_graph_capture(F):
    """Recorded into a CUDA graph the driver cannot stop early (the host reads
    no count): the graph holds all kmax steps and the matrices that met the
    rule stay as they are, so each replay reproduces the uncaptured call's
    iterates and step counts bit for bit."""
    xs = np.stack([W.sign_case(48, seed=320 + b, re_lo=0.05 + 0.4 * b, re_hi=0.5 + 0.6 * b)[0] for b in range(3)])
    m = torch.from_numpy(xs).cuda()
    eager = F.sign(m, eps=1e-10, kmax=40)
    want, want_steps = eager.out.cpu().numpy(), eager.steps()
    assert len(set(want_steps.tolist())) > 1 and max(want_steps) < 40
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up on the capture stream, outside the capture
        F.sign(m, eps=1e-10, kmax=40, check=False)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        r = F.sign(m, eps=1e-10, kmax=40, check=False)
    for _ in range(2):
        r.out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(r.steps(), want_steps)
        assert np.array_equal(r.out.cpu().numpy(), want)
