"""Pins for the CPU oracle (no GPU).

Each test checks the oracle against something other than itself: closed forms,
brute force, identities printed in the paper, LAPACK (via numpy) on inputs
where the result is unique, and invariants the paper proves.  Together they
catch a dropped term, a wrong sign, a wrong operand order or a transposed
operand anywhere in the oracle (see test_oracle_mutants.py).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import metrics
from paper_2208_01239_gb300 import flops
from paper_2208_01239_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U64 = 2.0 ** -53

ALL_GENERAL = {
    "cplx_lu_right": lambda o, m: o.cplx_lu_inv(m, left=False),
    "cplx_lu_left": lambda o, m: o.cplx_lu_inv(m, left=True),
    "frob_basic": lambda o, m: o.frob_inv_basic(m),
    "frob_lu": lambda o, m: o.frob_inv_lu(m),
    "frob_rand": lambda o, m: o.frob_inv_rand(m, 0.6180339887),
}


def _rand_complex(n, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))


def _golden_cases():
    cases, cur = [], None
    with open(os.path.join(GOLDEN, "special_inputs.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, _, val = line.partition(" ")
            if key == "name":
                cur = {"name": val}
                cases.append(cur)
            elif key == "n":
                cur["n"] = int(val)
            elif key in ("m", "inv"):
                if val == "SINGULAR":
                    cur[key] = None
                else:
                    vals = [complex(float(p.split(",")[0]), float(p.split(",")[1])) for p in val.split()]
                    cur[key] = np.array(vals).reshape(cur["n"], cur["n"])
            else:
                cur[key] = val
    return cases


# --------------------------------------------------------------------------- closed forms


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("name", sorted(ALL_GENERAL))
def test_2x2_closed_form(oracle_lib, name, seed):
    """[[a,b],[c,d]]^{-1} = (ad-bc)^{-1} [[d,-b],[-c,a]]."""
    m = _rand_complex(2, 100 + seed)
    a, b, c, d = m[0, 0], m[0, 1], m[1, 0], m[1, 1]
    expect = np.array([[d, -b], [-c, a]]) / (a * d - b * c)
    got = ALL_GENERAL[name](oracle.load(), m)
    assert metrics.forward_error(got, expect) < 1e-13


def test_integer_2x2_exact(oracle_lib):
    """[[1,2],[3,4]]^{-1} = [[-2,1],[3/2,-1/2]] exactly, also with an i shift."""
    m = np.array([[1, 2], [3, 4]], dtype=complex)
    expect = np.array([[-2, 1], [1.5, -0.5]], dtype=complex)
    for name, f in ALL_GENERAL.items():
        assert metrics.forward_error(f(oracle.load(), m), expect) < 1e-15, name
    assert np.array_equal(oracle.inv2x2(m), expect)
    assert np.allclose(oracle.adjugate_inv(m), expect, rtol=0, atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", range(4))
def test_adjugate_brute_force(oracle_lib, n, seed):
    """adj(M)/det(M) (Laplace expansion) agrees with every oracle route."""
    m = _rand_complex(n, 200 + 10 * n + seed)
    adj = oracle.adjugate_inv(m)
    assert metrics.res_right(m, adj) < 1e-14
    for name, f in ALL_GENERAL.items():
        assert metrics.forward_error(f(oracle.load(), m), adj) < 1e-12, name


@pytest.mark.parametrize("n", [1, 7, 33, 64])
def test_agrees_with_lapack(oracle_lib, n):
    """numpy.linalg.inv (LAPACK zgesv) is an independent route to M^{-1}."""
    m = _rand_complex(n, 300 + n)
    ref = np.linalg.inv(m)
    kappa = np.linalg.cond(m)
    for name, f in ALL_GENERAL.items():
        got = f(oracle.load(), m)
        assert metrics.forward_error(got, ref) < 50 * n * kappa * U64, name
        assert metrics.residual_fro(m, got) < 1e-14, name


@pytest.mark.parametrize("n", [8, 64])
def test_ill_conditioned_closed_form(oracle_lib, n):
    """A = I, B = Q N Q^T with N^2 = -s^2 I: S = (1 - s^2) I and
    M^{-1} = (I - iB)/(1 - s^2) (Sec. 3, Theorem "illcond2")."""
    m, minv = W.ill_conditioned(n, seed=30 + n)
    for name, f in ALL_GENERAL.items():
        got = f(oracle.load(), m)
        assert metrics.forward_error(got, minv) < 1e-8, name
    _x, (_x2, s, _sinv) = oracle.frob_inv_basic(m, stages=True)
    s2 = 1.0 - (1.0 - 1e-6) ** 2
    assert np.abs(s - s2 * np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("n", [2, 16, 48])
def test_i_plus_iq(oracle_lib, n):
    """(I + iQ)^{-1} = (I - iQ)(Q^2 + I)^{-1} for orthogonal Q (Sec. 3)."""
    g = np.random.default_rng(400 + n)
    q, _ = np.linalg.qr(g.standard_normal((n, n)))
    m = np.eye(n) + 1j * q
    expect = (np.eye(n) - 1j * q) @ np.linalg.inv(q @ q + np.eye(n))
    for name, f in ALL_GENERAL.items():
        assert metrics.forward_error(f(oracle.load(), m), expect) < 1e-11, name


@pytest.mark.parametrize("n", [5, 64])
def test_hpd_closed_form(oracle_lib, n):
    """M = Q diag(lam) Q^H has M^{-1} = Q diag(1/lam) Q^H."""
    ms, qs, lams = W.hpd(n, 2, seed=50 + n, return_parts=True)
    for t in range(2):
        exact = W.hpd_exact_inverse(qs[t], lams[t])
        kappa = lams[t].max() / lams[t].min()
        for name, got in [("cplx_chol", oracle.cplx_chol_inv(ms[t])), ("frob_chol", oracle.frob_inv_chol(ms[t])),
                          ("cplx_lu", oracle.cplx_lu_inv(ms[t])), ("frob_lu", oracle.frob_inv_lu(ms[t]))]:
            assert metrics.forward_error(got, exact) < 20 * n * kappa * U64, name
        # inverse of a Hermitian matrix is Hermitian
        x = oracle.frob_inv_chol(ms[t])
        assert np.abs(x - x.conj().T).max() < 1e-12 * np.abs(x).max()


def test_hpd_reads_lower_triangle_only(oracle_lib):
    m = W.hpd(24, 1, seed=9)[0]
    bad = m.copy()
    iu = np.triu_indices(24, 1)
    bad[iu] = 1e3 * (1 + 1j)
    bad[np.diag_indices(24)] += 7j  # imaginary part of the diagonal is ignored
    for f in (oracle.cplx_chol_inv, oracle.frob_inv_chol):
        assert np.array_equal(f(m), f(bad))


# --------------------------------------------------------------------------- identities


def test_frobenius_stage_identities(oracle_lib):
    """X2 = A^{-1}B, S = A + B A^{-1} B (Sec. 2, Lemma 2.3 with tau = 1), and
    A^{-1} B S^{-1} = (B + A B^{-1} A)^{-1} = S^{-1} B A^{-1} (Sec. 2,
    proof of Theorem "optimal inverse")."""
    n = 40
    m = _rand_complex(n, 500)
    a, b = m.real, m.imag
    x, (x2, s, sinv) = oracle.frob_inv_basic(m, stages=True)
    np.testing.assert_allclose(x2, np.linalg.solve(a, b), rtol=0, atol=1e-10 * np.abs(x2).max())
    np.testing.assert_allclose(s, a + b @ np.linalg.solve(a, b), rtol=0, atol=1e-10 * np.abs(s).max())
    z = -x.imag
    z1 = np.linalg.inv(b + a @ np.linalg.solve(b, a))
    z2 = sinv @ b @ np.linalg.inv(a)
    np.testing.assert_allclose(z, z1, rtol=0, atol=1e-10 * np.abs(z).max())
    np.testing.assert_allclose(z, z2, rtol=0, atol=1e-10 * np.abs(z).max())
    # the real 2n x 2n embedding [[A, -B], [B, A]] has the inverse
    # [[Re, -Im], [Im, Re]] of M^{-1} (Sec. 1.3)
    big = np.block([[a, -b], [b, a]])
    emb = np.block([[x.real, -x.imag], [x.imag, x.real]])
    assert np.abs(big @ emb - np.eye(2 * n)).max() < 1e-11


def test_hpd_invariants(oracle_lib):
    """For HPD M: A SPD, B skew, S = A + B A^{-1} B SPD (Sec. 4.3, Lemma
    "positive real part")."""
    m = W.hpd(32, 1, seed=12)[0]
    a, b = m.real, m.imag
    assert np.allclose(a, a.T) and np.allclose(b, -b.T)
    assert np.linalg.eigvalsh(a).min() > 0
    _x, (_x2, s, _sinv) = oracle.frob_inv_basic(m, stages=True)
    assert np.abs(s - s.T).max() < 1e-10 * np.abs(s).max()
    assert np.linalg.eigvalsh(0.5 * (s + s.T)).min() > 0


def test_left_and_right_inverse(oracle_lib):
    """Both variants of Algorithm LU1 are two-sided inverses to rounding."""
    m = _rand_complex(50, 600)
    for left in (False, True):
        x = oracle.cplx_lu_inv(m, left=left)
        assert metrics.res_left(m, x) < 1e-14 * 50
        assert metrics.res_right(m, x) < 1e-14 * 50


# --------------------------------------------------------------------------- special inputs


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_golden_special_inputs(oracle_lib, case):
    m = case["m"]
    if case["inv"] is None:
        for name, f in ALL_GENERAL.items():
            with pytest.raises(oracle.OracleError):
                f(oracle.load(), m)
        return
    for name in ("cplx_lu_right", "cplx_lu_left", "frob_rand"):
        got = ALL_GENERAL[name](oracle.load(), m)
        assert metrics.forward_error(got, case["inv"]) < 1e-15, name


def test_diag_1_i_needs_almost_sure_variant(oracle_lib):
    """diag(1, i): A = diag(1, 0) is singular, so plain Frobenius inversion
    fails at the second pivot; the almost sure variant succeeds (Sec. 4.2)."""
    m = np.diag([1.0, 1j])
    with pytest.raises(oracle.OracleError) as e:
        oracle.frob_inv_lu(m)
    assert e.value.info == 2
    with pytest.raises(oracle.OracleError):
        oracle.frob_inv_basic(m)
    for mu in (0.1, 0.5, 0.9):
        np.testing.assert_allclose(oracle.frob_inv_rand(m, mu), np.diag([1.0, -1j]), rtol=0, atol=1e-15)


def test_rand_lemma_bad_mu(oracle_lib):
    """A - mu B is singular for at most n values of mu (Sec. 4.2, Lemma
    "rand Frob"): here exactly mu = 0.5 and mu = 1."""
    a = np.diag([0.5, 1.0])
    b = np.eye(2)
    m = a + 1j * b
    for bad in (0.5, 1.0):
        with pytest.raises(oracle.OracleError):
            oracle.frob_inv_rand(m, bad)
    np.testing.assert_allclose(oracle.frob_inv_rand(m, 0.25), np.diag(1.0 / np.diag(m)), rtol=0, atol=1e-15)


def test_not_hpd_reported(oracle_lib):
    m = np.diag([1.0, -1.0, 2.0]).astype(complex)
    with pytest.raises(oracle.OracleError) as e:
        oracle.cplx_chol_inv(m)
    assert e.value.info == 2
    with pytest.raises(oracle.OracleError) as e:
        oracle.frob_inv_chol(m)
    assert e.value.info == 2


def test_nonfinite_input_reported(oracle_lib):
    m = _rand_complex(6, 700)
    m[3, 2] = np.nan
    for name, f in ALL_GENERAL.items():
        if name == "frob_basic":
            continue  # the NaN sits in column 2: A's LU meets it at step <= 3
        with pytest.raises(oracle.OracleError):
            f(oracle.load(), m)


# --------------------------------------------------------------------------- reporting model


def test_paper_flop_counts():
    """Counts stated in Sec. 4.1 and 4.3 (Propositions "Flop counts")."""
    with open(os.path.join(GOLDEN, "flop_counts.txt")) as f:
        rows = [ln.split(None, 3) for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 4
    for alg, num, den, _cite in rows:
        assert flops.PAPER[alg] == flops.F(int(num), int(den)), alg
    # the 22% HPD claim of Sec. 4.3 is the ratio 28/23 - 1
    assert abs(float(flops.PAPER["cplx_chol"] / flops.PAPER["frob_chol"]) - 1 - 0.2174) < 1e-3


def test_executed_flop_counts():
    assert flops.EXECUTED["frob_lu"] == flops.F(26, 3)
    assert flops.EXECUTED["cplx_lu"] == 8
    assert flops.EXECUTED["frob_chol"] == flops.F(19, 3)
    assert flops.EXECUTED["cplx_chol"] == 4
    assert flops.nominal(10) == 8000.0


# --------------------------------------------------------------------------- generators


def test_kappa_generator():
    """The Sec. 5.1 accuracy generator gives kappa(A) = kappa(B) = kappa."""
    m = W.kappa_controlled(40, 10.0, seed=3)
    assert abs(np.linalg.cond(m.real) - 10.0) < 1e-8
    assert abs(np.linalg.cond(m.imag) - 10.0) < 1e-8


def test_condition_of_real_embedding():
    """kappa(A + iB) equals kappa of [[A, -B], [B, A]] (Sec. 3)."""
    m = _rand_complex(20, 800)
    big = np.block([[m.real, -m.imag], [m.imag, m.real]])
    assert abs(np.linalg.cond(m) / np.linalg.cond(big) - 1) < 1e-10


def test_ill_conditioned_generator():
    """kappa(A) = kappa(B) = 1 but kappa(M) ~ 1/(1 - s) (Sec. 3)."""
    m, _ = W.ill_conditioned(32, seed=1)
    assert abs(np.linalg.cond(m.imag) - 1) < 1e-8
    kappa = np.linalg.cond(m)
    assert 1e5 < kappa < 1e7


# ------------------------------------------------------------------ formula for invertible B (Sec. 4.2)


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_frob_inv_b_adjugate(oracle_lib, n):
    g = np.random.default_rng(700 + n)
    m = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    assert metrics.forward_error(oracle.frob_inv_b(m), oracle.adjugate_inv(m)) <= 1e-12


def test_frob_inv_b_singular_real_part(oracle_lib):
    """A singular, B invertible: the A route fails at its last pivot, the B
    formula gives the inverse (LAPACK on the unique result)."""
    g = np.random.default_rng(71)
    n = 30
    a = g.standard_normal((n, n))
    a[:, 7] = 0.0
    m = a + 1j * g.standard_normal((n, n))
    with pytest.raises(oracle.OracleError):
        oracle.frob_inv_lu(m)
    assert metrics.forward_error(oracle.frob_inv_b(m), np.linalg.inv(m)) <= 1e-11


def test_frob_inv_b_is_frobenius_of_minus_i_m(oracle_lib):
    """(A + iB)^{-1} = -i (B - iA)^{-1}: the B formula equals -i times the A
    formula applied to B - iA."""
    g = np.random.default_rng(72)
    m = g.standard_normal((9, 9)) + 1j * g.standard_normal((9, 9))
    mp = m.imag - 1j * m.real
    assert np.abs(oracle.frob_inv_b(m) - (-1j) * oracle.frob_inv_basic(mp)).max() <= 1e-12 * np.abs(
        np.linalg.inv(m)).max()


# ------------------------------------------------------------------ bicomplex matrices (Sec. 2.4, m = 2)


def _bimul(a, b, c, d):
    """(A + jB)(C + jD) = (AC - BD) + j(AD + BC), j^2 = -1, j commuting with i."""
    return a @ c - b @ d, a @ d + b @ c


def test_bicomplex_scalar_closed_form(oracle_lib):
    """For commuting entries (a + jb)^{-1} = (a - jb) / (a^2 + b^2)."""
    for a, b in ((2.0 + 1j, -0.5 + 0.25j), (0.3 - 2j, 1.1 + 0j), (1j, 0.0)):
        y0, y1 = oracle.bicomplex_inv(np.array([[a]]), np.array([[b]]))
        d = a * a + b * b
        assert abs(y0[0, 0] - a / d) <= 1e-15 * abs(a / d) + 1e-300
        assert abs(y1[0, 0] + b / d) <= 1e-15 * max(abs(b / d), 1e-300)


@pytest.mark.parametrize("n", [2, 5, 17])
def test_bicomplex_product_is_identity(oracle_lib, n):
    g = np.random.default_rng(800 + n)
    a = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    b = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    y0, y1 = oracle.bicomplex_inv(a, b)
    for p0, p1 in (_bimul(a, b, y0, y1), _bimul(y0, y1, a, b)):
        assert np.abs(p0 - np.eye(n)).max() <= 1e-12 and np.abs(p1).max() <= 1e-12


def test_bicomplex_special_cases(oracle_lib):
    """B = 0: Y0 = A^{-1}, Y1 = 0; A = 0: (jB)^{-1} = -j B^{-1}."""
    g = np.random.default_rng(81)
    a = g.standard_normal((6, 6)) + 1j * g.standard_normal((6, 6))
    z = np.zeros_like(a)
    y0, y1 = oracle.bicomplex_inv(a, z)
    assert np.abs(y0 - np.linalg.inv(a)).max() <= 1e-12 * np.abs(np.linalg.inv(a)).max() and np.abs(y1).max() == 0.0
    y0, y1 = oracle.bicomplex_inv(z, a)
    assert np.abs(y0).max() <= 1e-13 and np.abs(y1 + np.linalg.inv(a)).max() <= 1e-12 * np.abs(np.linalg.inv(a)).max()


def test_executed_flop_counts():
    """The executed counts the benchmark reports: Frobenius inversion with LU
    26 n^3 / 3 (LU 2/3, two solves 2, product 2, LU 2/3, S^{-1} 4/3, product 2),
    complex LU inversion 8 n^3 (4 x (2/3 + 4/3)), Frobenius-Cholesky 19 n^3 / 3;
    and the paper's 28/3 and 32/3 (Sec. 4.1)."""
    from fractions import Fraction
    assert flops.EXECUTED["frob_lu"] == Fraction(26, 3)
    assert flops.EXECUTED["cplx_lu"] == 8
    assert flops.EXECUTED["frob_chol"] == Fraction(19, 3)
    assert flops.PAPER["frob_lu"] == Fraction(28, 3) and flops.PAPER["cplx_lu"] == Fraction(32, 3)


def test_bench_roofline_arithmetic():
    """The benchmark's roofline picks the kernel variant with the most device
    time per step and divides its algorithmic flops by that time."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench_mod", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    prof = {"a": (3.0, 10.0, 1.0e10), "b": (1.0, 30.0, 3.3e10), "c": (5.0, 2.0, 0.0)}
    r = bench._roofline(prof, {"sm_mhz": 1035.0})
    assert r["kernel"] == "b"
    assert abs(r["achieved"] - 3.3e10 / 30e-3 / 1e12) < 1e-12
    assert abs(r["frac"] - r["achieved"] / bench.FP64_PEAK_TFLOPS) < 1e-12
    assert abs(r["peak_at_sampled_clock"] - bench.FP64_PEAK_TFLOPS / 2) < 1e-9
    assert abs(r["share_of_step"] - 30.0 / 42.0) < 1e-12


def test_bench_roofline_digit_products():
    """When the FP64 digit-product GEMM dominates, the roofline is the tensor
    pipe's: its FP64 flops times the 36 BF16 digit products each takes,
    against the BF16 peak."""
    import importlib.util
    import os
    spec = importlib.util.spec_from_file_location(
        "bench_mod", os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    prof = {"ozr_gemm<f64 digits>": (10.0, 100.0, 2.0e12), "gemm<f64,op0,op0,axpby>": (5.0, 50.0, 5e10)}
    r = bench._roofline(prof, {"sm_mhz": 2070.0})
    assert r["bound"] == "tensor" and r["kernel"] == "ozr_gemm<f64 digits>"
    assert abs(r["achieved"] - 36 * 2.0e12 / 0.1 / 1e12) < 1e-9
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
