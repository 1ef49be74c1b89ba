"""The C-ABI library builds, loads and exports every function that
include/frobinv.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "frobinv.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "while", "sizeof")))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_01239_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_entry_points():
    names = _declared_functions()
    for required in ("frob_inv", "frob_inv_hpd", "cplx_lu_inv", "cplx_chol_inv", "frob_workspace_bytes",
                     "frob_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), f"libfrobinv.so does not export {name}"


def test_host_only_calls(lib):
    """Calls that touch no device: sizes, status strings, argument checks."""
    lib.frob_workspace_bytes.restype = ctypes.c_size_t
    lib.frob_workspace_bytes.argtypes = [ctypes.c_int] * 4
    assert lib.frob_workspace_bytes(0, 256, 1, 0) > 5 * 256 * 256 * 8
    assert lib.frob_workspace_bytes(0, 0, 1, 0) == 0
    assert lib.frob_workspace_bytes(9, 16, 1, 0) == 0
    # fp32 planes are half the size of fp64 planes
    # FP32 planes are half the size (below order 256, where FP32 products
    # need no split-TF32 scratch)
    assert lib.frob_workspace_bytes(1, 128, 4, 1) < lib.frob_workspace_bytes(1, 128, 4, 0)
    # the FP64 general route reserves the digit-product scratch from order 256 on
    assert lib.frob_workspace_bytes(0, 256, 1, 0) > lib.frob_workspace_bytes(0, 255, 1, 0) + 2 * 8 * 256 * 256 * 2
    lib.frob_status_str.restype = ctypes.c_char_p
    assert lib.frob_status_str(2) == b"FROB_ERR_SINGULAR"
    # argument errors return synchronously, before any launch
    lib.frob_inv.restype = ctypes.c_int
    vp = ctypes.c_void_p
    lib.frob_inv.argtypes = [ctypes.c_int, ctypes.c_int, vp, ctypes.c_int64, ctypes.c_int64, vp, ctypes.c_int64,
                             ctypes.c_int64, vp, vp, ctypes.c_size_t, vp, vp]
    assert lib.frob_inv(0, 1, 16, 1, 1, 4096, 1, 1, None, 256, 1 << 20, 512, None) == 1      # n < 1
    assert lib.frob_inv(4, 1, 16, 3, 16, 4096, 4, 16, None, 256, 1 << 20, 512, None) == 1     # ldm < n
    assert lib.frob_inv(4, 1, None, 4, 16, 4096, 4, 16, None, 256, 1 << 20, 512, None) == 1   # NULL input
    assert lib.frob_inv(4, 1, 4096, 4, 16, 4096, 4, 16, None, 256, 1 << 20, 512, None) == 1   # in == out
    assert lib.frob_inv(4, 1, 16, 4, 16, 4096, 4, 16, None, 256, 8, 512, None) == 7          # ws too small
    assert lib.frob_inv(4, 1, 16, 4, 16, 4096, 4, 16, None, 257, 1 << 20, 512, None) == 7    # misaligned ws


def test_opts_layout_matches_the_binding():
    """frob_opts is 40 bytes (prec, almost_sure, seed, attempt, ns_max_iter,
    ns_tol, part, fp64_gemm); the binding's ctypes mirror has the same size
    and offsets."""
    from paper_2208_01239_gb300 import frob
    o = frob.FrobOpts
    assert ctypes.sizeof(o) == 40
    assert [o.seed.offset, o.ns_tol.offset, o.part.offset, o.fp64_gemm.offset] == [8, 24, 32, 36]


def test_host_only_checks_of_the_newer_entry_points(lib):
    """Argument and workspace errors of the part option, the Newton drivers,
    the bicomplex inverse and the augmented solve return synchronously,
    before any launch (no GPU is touched)."""
    from paper_2208_01239_gb300 import frob
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
    L = ctypes.CDLL(frob.library_path())
    # frob_inv: part out of range, an unknown fp64_gemm, part with the almost sure option
    L.frob_inv.restype = i32
    L.frob_inv.argtypes = [i32, i32, vp, i64, i64, vp, i64, i64, ctypes.POINTER(frob.FrobOpts), vp, sz, vp, vp]
    for part, gemm, almost in ((3, 0, 0), (0, 2, 0), (0, -1, 0), (1, 0, 1), (2, 0, 1)):
        o = frob._opts("fp64", part="A")
        o.part, o.fp64_gemm, o.almost_sure = part, gemm, almost
        assert L.frob_inv(4, 1, 16, 4, 16, 4096, 4, 16, ctypes.byref(o), 256, 1 << 20, 512, None) == 1
    # workspace sizes
    L.frob_newton_workspace_bytes.restype = sz
    L.frob_newton_workspace_bytes.argtypes = [i32, i32, i32, i32]
    assert L.frob_newton_workspace_bytes(64, 2, 0, 0) > 2 * 64 * 64 * 16
    assert L.frob_newton_workspace_bytes(64, 2, 0, 2) == 0          # no such route
    assert L.frob_newton_workspace_bytes(64, 2, 3, 1) == 0          # mixed with the complex-LU route
    assert L.frob_newton_workspace_bytes(600, 1, 3, 0) == 0         # mixed needs n <= 512
    L.frob_solve_workspace_bytes.restype = sz
    L.frob_solve_workspace_bytes.argtypes = [i32] * 5
    assert L.frob_solve_workspace_bytes(2, 64, 1, 1, 0) >= 4 * 64 * 64 * 8  # the 2n x 2n real matrix
    assert L.frob_solve_workspace_bytes(3, 64, 1, 1, 0) == 0
    L.frob_inv_bicomplex_workspace_bytes.restype = sz
    L.frob_inv_bicomplex_workspace_bytes.argtypes = [i32, i32, i32]
    assert L.frob_inv_bicomplex_workspace_bytes(32, 1, 0) > L.frob_inv_bicomplex_workspace_bytes(32, 1, 1)
    # frob_newton: bad kind, bad route, negative kmax, NaN eps, overlapping M / X, small workspace
    L.frob_newton.restype = i32
    L.frob_newton.argtypes = [i32, i32, i32, i32, vp, i64, i64, vp, i64, i64, vp, ctypes.c_double, i32, vp, sz, vp,
                              vp, vp]
    args = lambda kind=0, route=0, kmax=10, eps=1e-3, m=4096, x=1 << 20, ws=1 << 24, wsb=1 << 30: (
        kind, route, 8, 1, m, 8, 64, x, 8, 64, None, eps, kmax, ws, wsb, 256, 512, None)
    assert L.frob_newton(*args(kind=2)) == 1
    assert L.frob_newton(*args(route=5)) == 1
    assert L.frob_newton(*args(kmax=-1)) == 1
    assert L.frob_newton(*args(eps=float("nan"))) == 1
    assert L.frob_newton(*args(x=4096 + 16)) == 1                  # X overlaps M (and is not M itself)
    assert L.frob_newton(*args(wsb=64)) == 7
    # frob_sylvester: Lyapunov with p != q
    L.frob_sylvester.restype = i32
    L.frob_sylvester.argtypes = [i32, i32, i32, i32, vp, i64, i64, vp, i64, i64, i32, vp, i64, i64, vp, i64, i64,
                                 vp, ctypes.c_double, i32, vp, sz, vp, vp, vp]
    assert L.frob_sylvester(0, 4, 5, 1, 4096, 4, 16, None, 5, 25, 1, 1 << 16, 5, 20, 1 << 20, 5, 20, None, 0.1, 10,
                            1 << 24, 1 << 30, 256, 512, None) == 1
    # frob_polar: Q overlapping X
    L.frob_polar.restype = i32
    L.frob_polar.argtypes = [i32, i32, i32, vp, i64, i64, vp, i64, i64, vp, i64, i64, vp, ctypes.c_double, i32, vp,
                             sz, vp, vp, vp]
    assert L.frob_polar(0, 8, 1, 4096, 8, 64, 4096 + 32, 8, 64, 1 << 20, 8, 64, None, 1e-3, 10, 1 << 24, 1 << 30,
                        256, 512, None) == 1
    # frob_inv_bicomplex: Y0 overlapping Y1, and the part option
    L.frob_inv_bicomplex.restype = i32
    L.frob_inv_bicomplex.argtypes = [i32, i32, vp, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64,
                                     ctypes.POINTER(frob.FrobOpts), vp, sz, vp, vp]
    assert L.frob_inv_bicomplex(8, 1, 4096, 8, 64, 1 << 16, 8, 64, 1 << 20, 8, 64, (1 << 20) + 64, 8, 64, None,
                                1 << 24, 1 << 30, 512, None) == 1
    o = frob._opts("fp64", part="B")
    assert L.frob_inv_bicomplex(8, 1, 4096, 8, 64, 1 << 16, 8, 64, 1 << 20, 8, 64, 1 << 21, 8, 64, ctypes.byref(o),
                                1 << 24, 1 << 30, 512, None) == 1


def test_bindings_reject_bad_inputs_before_calling_the_library():
    """The Python binding's own checks (host tensors, dtypes, shapes, option
    names) raise before anything reaches the library; no GPU needed."""
    import torch
    from paper_2208_01239_gb300 import frob
    cpu = torch.zeros((4, 4), dtype=torch.complex128)
    with pytest.raises(TypeError):
        frob.sign(cpu)
    with pytest.raises(TypeError):
        frob.polar(cpu)
    with pytest.raises(TypeError):
        frob.sylvester(cpu, cpu, cpu)
    with pytest.raises(TypeError):
        frob.frob_inv_bicomplex(cpu, cpu)
    with pytest.raises(KeyError):
        frob._opts("fp64", part="C")
    assert frob.ROUTE == {"frob": 0, "cplx_lu": 1} and frob.PART == {"A": 0, "B": 1, "auto": 2}
    o = frob._opts("fp32", part="auto")
    assert (o.prec, o.part, o.fp64_gemm, o.almost_sure) == (frob.PREC["fp32"], 2, 0, 0)


def test_batched_plan_sizes(lib):
    """The uneven-batch planner (host only): buckets of order 32 ceil(n/32);
    a list whose orders share a bucket needs less workspace than the same
    count spread over more buckets' worth of padding; an order < 1 or more
    than 64 distinct buckets is refused (0); the mixed precisions need
    n <= 512."""
    import numpy as np
    i32, sz, vp = ctypes.c_int, ctypes.c_size_t, ctypes.c_void_p
    f = lib.frob_inv_batched_workspace_bytes
    f.restype = sz
    f.argtypes = [i32, i32, vp, i32]

    def ws(ns, op=0, prec=0):
        a = np.ascontiguousarray(np.array(ns, dtype=np.int32))
        return f(op, len(ns), a.ctypes.data, prec)

    assert ws([33, 40, 64]) > 0
    assert ws([33, 40, 64]) == ws([64, 64, 64])                           # one bucket of order 64 either way
    assert ws([31, 33]) < ws([31, 65])                                    # buckets 32 + 64 vs 32 + 96
    assert ws([0, 5]) == 0
    assert ws([32 * k for k in range(1, 66)]) == 0                        # 65 distinct buckets
    assert ws([32 * k for k in range(1, 65)]) > 0                         # 64 are allowed
    assert ws([600], prec=3) == 0 and ws([500], prec=3) > 0               # mixed: n <= 512
    assert ws([500], op=2, prec=3) > 0 and ws([500], op=3, prec=3) > 0    # the complex refined controls
    assert ws([500], prec=2) == 0                                         # FROB_MIXED_TF32: unsupported
    assert ws([10], op=7) == 0


def test_autotune_cache_host_side():
    """The split autotuner's cache is empty until a tuned call runs, and
    clearing it is a host operation."""
    from paper_2208_01239_gb300 import frob
    frob.autotune_clear()
    assert frob.autotune_report() == {}
    frob.autotune(True)
    frob.autotune(False)
    assert frob.autotune_report() == {}
