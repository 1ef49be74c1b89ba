"""Thin ctypes binding over libfrobinv.so (the C ABI in include/frobinv.h).

Argument marshalling only: every step of the inversion runs in the CUDA
kernels of the library.  PyTorch supplies device memory and the current
stream.  There is no CPU fallback: if the library is missing or no CUDA
device is present, the calls raise.

The entry points keep the C names:

* :func:`frob_inv`       Frobenius inversion (Sec. 4.1; almost sure variant
                         of Sec. 4.2 with ``almost_sure=True``)
* :func:`frob_inv_hpd`   Frobenius inversion of HPD matrices (Sec. 4.3)
* :func:`cplx_lu_inv`    complex LU inversion baseline (Sec. 4)
* :func:`cplx_chol_inv`  complex Cholesky inversion baseline (Sec. 4.3)

Each takes a complex tensor of shape (n, n) or (batch, n, n), complex128 for
``prec="fp64"`` and complex64 for ``prec="fp32"``, on the GPU or on the host
(host tensors are copied to the device and the result back).
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

import numpy as np
import torch

from . import build as _build

FROB_OK = 0
FROB_ERR_ARG = 1
FROB_ERR_SINGULAR = 2
FROB_ERR_NOT_HPD = 3
FROB_ERR_NOT_CONVERGED = 4
FROB_ERR_TIMEOUT = 5
FROB_ERR_CUDA = 6
FROB_ERR_WORKSPACE = 7
FROB_ERR_UNSUPPORTED = 8

PREC = {"fp64": 0, "fp32": 1, "mixed_tf32": 2, "mixed_bf16": 3}
OP = {"frob_inv": 0, "frob_inv_hpd": 1, "cplx_lu_inv": 2, "cplx_chol_inv": 3, "frob_inv_adjoint": 4}

INFO_DTYPE = np.dtype([("status", "<i4"), ("bad_index", "<i4"), ("ns_iters", "<i4"), ("fell_back", "<i4"),
                       ("mu", "<f8"), ("residual", "<f8")])
assert INFO_DTYPE.itemsize == 32


class FrobOpts(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int32), ("almost_sure", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("attempt", ctypes.c_int32), ("ns_max_iter", ctypes.c_int32), ("ns_tol", ctypes.c_double),
                ("part", ctypes.c_int32), ("fp64_gemm", ctypes.c_int32)]


PART = {"A": 0, "B": 1, "auto": 2}


class FrobError(RuntimeError):
    """Raised for a non-OK status; ``status`` is the frob_status code and
    ``info`` (if any) the per-matrix records."""

    def __init__(self, msg, status, info=None):
        super().__init__(msg)
        self.status = status
        self.info = info


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libfrobinv.so (built by ``paper_2208_01239_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libfrobinv.so is not built ({path}); run python -m paper_2208_01239_gb300.build")
        lib = ctypes.CDLL(path)
        vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        lib.frob_workspace_bytes.argtypes = [i32, i32, i32, i32]
        lib.frob_workspace_bytes.restype = sz
        common = [i32, i32, vp, i64, i64, vp, i64, i64]
        for name in ("frob_inv", "frob_inv_hpd"):
            f = getattr(lib, name)
            f.argtypes = common + [ctypes.POINTER(FrobOpts), vp, sz, vp, vp]
            f.restype = i32
        for name in ("cplx_lu_inv", "cplx_chol_inv"):
            f = getattr(lib, name)
            f.argtypes = common + [i32, vp, sz, vp, vp]
            f.restype = i32
        lib.cplx_inv_mixed.argtypes = [i32] + common + [ctypes.POINTER(FrobOpts), vp, sz, vp, vp]
        lib.cplx_inv_mixed.restype = i32
        lib.frob_status_str.argtypes = [i32]
        lib.frob_status_str.restype = ctypes.c_char_p
        lib.frob_version.argtypes = []
        lib.frob_version.restype = ctypes.c_char_p
        lib.frob_kernel_launches.argtypes = []
        lib.frob_kernel_launches.restype = ctypes.c_uint64
        lib.frob_inv_adjoint.argtypes = common + [vp, i64, i64, i32, vp, sz, vp]
        lib.frob_inv_adjoint.restype = i32
        lib.frob_inv_batched_workspace_bytes.argtypes = [i32, i32, vp, i32]
        lib.frob_inv_batched_workspace_bytes.restype = sz
        lib.frob_inv_batched.argtypes = [i32, i32, vp, vp, vp, vp, vp, vp, ctypes.POINTER(FrobOpts), vp, sz, vp, vp]
        lib.frob_inv_batched.restype = i32
        lib.frob_solve_workspace_bytes.argtypes = [i32, i32, i32, i32, i32]
        lib.frob_solve_workspace_bytes.restype = sz
        for name in ("frob_solve", "cplx_lu_solve", "aug_real_solve"):
            f = getattr(lib, name)
            f.argtypes = [i32, i32, i32, vp, i64, i64, vp, i64, i64, vp, i64, i64, i32, vp, sz, vp, vp]
            f.restype = i32
        lib.frob_gemm_tc.argtypes = [i32, i32, i32, i32, i32, vp, i64, i64, vp, i64, i64, vp, i64, i64, vp, sz, vp,
                                     vp]
        lib.frob_gemm_tc.restype = i32
        lib.frob_gemm_tc_workspace_bytes.argtypes = [i32, i32, i32, i32, i32]
        lib.frob_gemm_tc_workspace_bytes.restype = sz
        lib.frob_gemm_f64.argtypes = [i32, i32, i32, i32, vp, i64, i64, i32, vp, i64, i64, i32, vp, i64, i64,
                                      ctypes.c_double, ctypes.c_double, vp, sz, vp, vp]
        lib.frob_gemm_f64.restype = i32
        lib.frob_gemm_f64_workspace_bytes.argtypes = [i32, i32, i32, i32]
        lib.frob_gemm_f64_workspace_bytes.restype = sz
        lib.frob_newton_workspace_bytes.argtypes = [i32, i32, i32, i32]
        lib.frob_newton_workspace_bytes.restype = sz
        lib.frob_polar_workspace_bytes.argtypes = [i32, i32, i32, i32]
        lib.frob_polar_workspace_bytes.restype = sz
        lib.frob_sylvester_workspace_bytes.argtypes = [i32, i32, i32, i32, i32]
        lib.frob_sylvester_workspace_bytes.restype = sz
        dbl = ctypes.c_double
        lib.frob_newton.argtypes = [i32, i32, i32, i32, vp, i64, i64, vp, i64, i64, ctypes.POINTER(FrobOpts), dbl,
                                    i32, vp, sz, vp, vp, vp]
        lib.frob_newton.restype = i32
        lib.frob_polar.argtypes = [i32, i32, i32, vp, i64, i64, vp, i64, i64, vp, i64, i64, ctypes.POINTER(FrobOpts),
                                   dbl, i32, vp, sz, vp, vp, vp]
        lib.frob_polar.restype = i32
        lib.frob_sylvester.argtypes = [i32, i32, i32, i32, vp, i64, i64, vp, i64, i64, i32, vp, i64, i64, vp, i64, i64,
                                       ctypes.POINTER(FrobOpts), dbl, i32, vp, sz, vp, vp, vp]
        lib.frob_sylvester.restype = i32
        lib.frob_inv_bicomplex_workspace_bytes.argtypes = [i32, i32, i32]
        lib.frob_inv_bicomplex_workspace_bytes.restype = sz
        lib.frob_inv_bicomplex.argtypes = [i32, i32, vp, i64, i64, vp, i64, i64, vp, i64, i64, vp, i64, i64,
                                           ctypes.POINTER(FrobOpts), vp, sz, vp, vp]
        lib.frob_inv_bicomplex.restype = i32
        lib.frob_autotune_enable.argtypes = [i32]
        lib.frob_autotune_enable.restype = None
        lib.frob_autotune_clear.argtypes = []
        lib.frob_autotune_clear.restype = None
        lib.frob_autotune_report.argtypes = [ctypes.c_char_p, sz]
        lib.frob_autotune_report.restype = sz
        lib.frob_profile_enable.argtypes = [i32]
        lib.frob_profile_enable.restype = None
        lib.frob_profile_report.argtypes = [ctypes.c_char_p, sz]
        lib.frob_profile_report.restype = sz
        _lib = lib
        return lib


def autotune(on: bool = True):
    """Turn the autotuning of the stream split on or off (see
    frob_autotune_enable in include/frobinv.h)."""
    load().frob_autotune_enable(1 if on else 0)


def autotune_clear():
    load().frob_autotune_clear()


def autotune_report() -> dict:
    """{(op, prec, n, batch): (slices, ms_one_slice, ms_two_slices)}."""
    lib = load()
    need = int(lib.frob_autotune_report(None, 0))
    buf = ctypes.create_string_buffer(need)
    lib.frob_autotune_report(buf, need)
    raw = json.loads(buf.value.decode())
    return {tuple(int(v) for v in k.split(",")): (int(x[0]), float(x[1]), float(x[2])) for k, x in raw.items()}


def profile_enable(on: bool = True):
    """Start (discarding earlier records) or stop per-kernel event timing."""
    load().frob_profile_enable(1 if on else 0)


def profile_report() -> dict:
    """{kernel variant: (launches, total device ms, algorithmic flops)} since
    profile_enable (flops 0 for kernels that do not count them)."""
    import json
    lib = load()
    buf = ctypes.create_string_buffer(1 << 20)
    need = int(lib.frob_profile_report(buf, len(buf)))
    if need > len(buf):
        raise RuntimeError("profile report truncated")
    return {k: (int(v[0]), float(v[1]), float(v[2]) if len(v) > 2 else 0.0)
            for k, v in json.loads(buf.value.decode()).items()}


def status_str(code: int) -> str:
    return load().frob_status_str(int(code)).decode()


def workspace_bytes(op: str, n: int, batch: int, prec: str = "fp64") -> int:
    return int(load().frob_workspace_bytes(OP[op], n, batch, PREC[prec]))


def _cdtype(prec: str):
    return torch.complex64 if prec == "fp32" else torch.complex128


def parse_info(info: torch.Tensor) -> np.ndarray:
    """Device info records -> numpy structured array (synchronises)."""
    return info.cpu().numpy().view(INFO_DTYPE).reshape(-1)


def check_info(info_np: np.ndarray, what: str):
    bad = np.nonzero(info_np["status"] != FROB_OK)[0]
    if len(bad):
        b = int(bad[0])
        st = int(info_np["status"][b])
        raise FrobError(f"{what}: matrix {b}: {status_str(st)} (bad_index={int(info_np['bad_index'][b])}); "
                        f"{len(bad)} of {len(info_np)} matrices failed", st, info_np)


class Result:
    """Output of a call: the inverse and the device-side info records."""

    def __init__(self, x: torch.Tensor, info: torch.Tensor):
        self.x = x
        self.info_dev = info

    def info(self) -> np.ndarray:
        return parse_info(self.info_dev)


def _call(op: str, m: torch.Tensor, prec: str, opts: FrobOpts | None, out: torch.Tensor | None,
          ws: torch.Tensor | None, info: torch.Tensor | None, check: bool) -> Result:
    lib = load()
    on_host = not m.is_cuda
    if on_host:
        m = m.pin_memory().to("cuda", non_blocking=True) if torch.cuda.is_available() else m.cuda()
    if m.dtype != _cdtype(prec):
        raise TypeError(f"{op}: expected {_cdtype(prec)} for prec={prec}, got {m.dtype}")
    squeeze = m.dim() == 2
    m3 = m.unsqueeze(0) if squeeze else m
    if m3.dim() != 3 or m3.shape[-1] != m3.shape[-2]:
        raise ValueError(f"{op}: expected (n, n) or (batch, n, n), got {tuple(m.shape)}")
    if m3.stride(-1) != 1:
        m3 = m3.contiguous()
    batch, n = m3.shape[0], m3.shape[-1]
    dev = m3.device
    if out is None:
        out3 = torch.empty((batch, n, n), dtype=m3.dtype, device=dev)
    else:
        out3 = out.unsqueeze(0) if out.dim() == 2 else out
    need = int(lib.frob_workspace_bytes(OP[op], n, batch, PREC[prec]))
    if ws is None:
        ws = torch.empty(need + 256, dtype=torch.uint8, device=dev)
    base = ws.data_ptr()
    pad = (-base) % 256
    ws_ptr, ws_bytes = base + pad, ws.numel() - pad
    if info is None:
        info = torch.zeros((batch, 32), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    args = (n, batch, m3.data_ptr(), m3.stride(1), m3.stride(0), out3.data_ptr(), out3.stride(1), out3.stride(0))
    with torch.cuda.device(dev):
        if op in ("frob_inv", "frob_inv_hpd"):
            st = getattr(lib, op)(*args, ctypes.byref(opts) if opts is not None else None, ws_ptr, ws_bytes,
                                  info.data_ptr(), stream)
        elif opts is not None:  # the complex inverses' refined control (cplx_inv_mixed)
            st = lib.cplx_inv_mixed(OP[op], *args, ctypes.byref(opts), ws_ptr, ws_bytes, info.data_ptr(), stream)
        else:
            st = getattr(lib, op)(*args, PREC[prec], ws_ptr, ws_bytes, info.data_ptr(), stream)
    if st != FROB_OK:
        raise FrobError(f"{op}: {status_str(st)}", st)
    res = Result(out3[0] if (squeeze and out is None) else (out if out is not None else out3), info)
    if check:
        check_info(res.info(), op)
    if on_host:
        res.x = res.x.cpu()
    return res


GEMM = {"auto": 0, "fp64_pipe": 1}


def _opts(prec: str, almost_sure: bool = False, seed: int = 0, attempt: int = 0, ns_tol: float = 1e-14,
          ns_max_iter: int = 8, part: str = "A", gemm: str = "auto") -> FrobOpts:
    o = FrobOpts()
    o.part = PART[part]
    o.fp64_gemm = GEMM[gemm]
    o.prec = PREC[prec]
    o.almost_sure = 1 if almost_sure else 0
    o.seed = seed
    o.attempt = attempt
    o.ns_max_iter = ns_max_iter
    o.ns_tol = ns_tol
    return o


def frob_inv(m: torch.Tensor, prec: str = "fp64", almost_sure: bool = False, seed: int = 0, attempt: int = 0,
             out=None, ws=None, info=None, check: bool = True, ns_tol: float = 1e-14, ns_max_iter: int = 8,
             part: str = "A", gemm: str = "auto") -> Result:
    """(A + iB)^{-1} = S^{-1} - i A^{-1} B S^{-1}, S = A + B A^{-1} B.

    part: "A" (the formula above), "B" (the formula for invertible B,
    B^{-1}A(AB^{-1}A + B)^{-1} - i(AB^{-1}A + B)^{-1}, Sec. 4.2) or "auto"
    (per matrix, the real part whose LU has the larger pivot ratio).
    gemm (FP64): "auto" runs products of at least 256 in every dimension as
    exact digit products on the BF16 tensor cores, "fp64_pipe" keeps every
    product on the FP64 pipe.
    ns_tol / ns_max_iter: stopping rule of the mixed precisions' Newton-Schulz
    refinement (relative residual ||I - M X||_F / (||M||_F ||X||_F))."""
    return _call("frob_inv", m, prec, _opts(prec, almost_sure, seed, attempt, ns_tol, ns_max_iter, part, gemm), out,
                 ws, info, check)


def frob_inv_hpd(m: torch.Tensor, prec: str = "fp64", out=None, ws=None, info=None, check: bool = True,
                 ns_tol: float = 1e-14, ns_max_iter: int = 8, gemm: str = "auto") -> Result:
    """Frobenius inversion with two real Cholesky factorisations (HPD input,
    lower triangle read); gemm as for frob_inv."""
    return _call("frob_inv_hpd", m, prec, _opts(prec, ns_tol=ns_tol, ns_max_iter=ns_max_iter, gemm=gemm), out, ws,
                 info, check)


def cplx_lu_inv(m: torch.Tensor, prec: str = "fp64", out=None, ws=None, info=None, check: bool = True,
                ns_tol: float = 1e-14, ns_max_iter: int = 8) -> Result:
    """Complex LU inversion with partial pivoting (baseline).  prec
    "mixed_bf16": the control for the mixed Frobenius form, an FP32 complex-LU
    start with the same Newton-Schulz refinement (cplx_inv_mixed)."""
    opts = _opts(prec, ns_tol=ns_tol, ns_max_iter=ns_max_iter) if prec.startswith("mixed") else None
    return _call("cplx_lu_inv", m, prec, opts, out, ws, info, check)


def cplx_chol_inv(m: torch.Tensor, prec: str = "fp64", out=None, ws=None, info=None, check: bool = True,
                  ns_tol: float = 1e-14, ns_max_iter: int = 8) -> Result:
    """Complex Cholesky inversion (HPD baseline, lower triangle read); prec
    "mixed_bf16" as for cplx_lu_inv."""
    opts = _opts(prec, ns_tol=ns_tol, ns_max_iter=ns_max_iter) if prec.startswith("mixed") else None
    return _call("cplx_chol_inv", m, prec, opts, out, ws, info, check)


class Batched:
    """A preallocated call of frob_inv_batched for a fixed list of orders.

    ``inputs[i]`` / ``outputs[i]`` are (n_i, n_i) device tensors owned by the
    plan; fill the inputs, then :meth:`run`.  :meth:`run` launches a fixed
    kernel sequence on the current stream with no allocation, so it can be
    captured with ``torch.cuda.graph`` after one eager call."""

    def __init__(self, ns, op: str = "frob_inv", prec: str = "fp64", device="cuda", ns_tol: float = 1e-14,
                 ns_max_iter: int = 8, part: str = "A"):
        lib = load()
        self.lib = lib
        self.ns = [int(n) for n in ns]
        self.batch = len(self.ns)
        self.op = OP[op]
        self.prec = prec
        dt = _cdtype(prec)
        dev = torch.device(device)
        self.n_host = np.ascontiguousarray(np.array(self.ns, dtype=np.int32))
        self.n_dev = torch.tensor(self.ns, dtype=torch.int32, device=dev)
        self.inputs = [torch.zeros((n, n), dtype=dt, device=dev) for n in self.ns]
        self.outputs = [torch.zeros((n, n), dtype=dt, device=dev) for n in self.ns]
        self.m_ptrs = torch.tensor([t.data_ptr() for t in self.inputs], dtype=torch.int64, device=dev)
        self.x_ptrs = torch.tensor([t.data_ptr() for t in self.outputs], dtype=torch.int64, device=dev)
        self.lds = torch.tensor(self.ns, dtype=torch.int64, device=dev)
        need = int(lib.frob_inv_batched_workspace_bytes(self.op, self.batch, self.n_host.ctypes.data, PREC[prec]))
        if need == 0:
            raise FrobError("frob_inv_batched: unsupported sizes / precision / operation", FROB_ERR_UNSUPPORTED)
        self.ws = torch.empty(need + 256, dtype=torch.uint8, device=dev)
        self.pad = (-self.ws.data_ptr()) % 256
        self.info_dev = torch.zeros((self.batch, 32), dtype=torch.uint8, device=dev)
        self.opts = _opts(prec, part=part)
        self.opts.ns_tol = ns_tol
        self.opts.ns_max_iter = ns_max_iter

    def run(self):
        st = self.lib.frob_inv_batched(self.op, self.batch, self.n_host.ctypes.data, self.n_dev.data_ptr(),
                                       self.m_ptrs.data_ptr(), self.lds.data_ptr(), self.x_ptrs.data_ptr(),
                                       self.lds.data_ptr(), ctypes.byref(self.opts), self.ws.data_ptr() + self.pad,
                                       self.ws.numel() - self.pad, self.info_dev.data_ptr(),
                                       torch.cuda.current_stream(self.ws.device).cuda_stream)
        if st != FROB_OK:
            raise FrobError(f"frob_inv_batched: {status_str(st)}", st)

    def info(self) -> np.ndarray:
        return parse_info(self.info_dev)


def frob_inv_batched(mats, op: str = "frob_inv", prec: str = "fp64", check: bool = True, part: str = "A"):
    """Invert a list of square complex matrices of different orders in one
    call; returns (list of inverses, info records).  ``part`` as for
    :func:`frob_inv` (op "frob_inv" only)."""
    plan = Batched([m.shape[-1] for m in mats], op=op, prec=prec,
                   device=mats[0].device if mats[0].is_cuda else "cuda", part=part)
    for dst, src in zip(plan.inputs, mats):
        dst.copy_(src)
    plan.run()
    info = plan.info()
    if check:
        check_info(info, "frob_inv_batched")
    return plan.outputs, info


def _solve(name: str, op: int, m: torch.Tensor, rhs: torch.Tensor, prec: str, check: bool) -> Result:
    lib = load()
    on_host = not m.is_cuda
    if on_host:
        m, rhs = m.cuda(), rhs.cuda()
    if m.dtype != _cdtype(prec) or rhs.dtype != m.dtype:
        raise TypeError(f"{name}: expected {_cdtype(prec)} for prec={prec}")
    m3 = m if m.dim() == 3 else m.unsqueeze(0)
    r = rhs
    if r.dim() == m.dim() - 1:
        r = r.unsqueeze(-1)
    r3 = r if r.dim() == 3 else r.unsqueeze(0)
    m3, r3 = m3.contiguous(), r3.contiguous()
    batch, n, nrhs = m3.shape[0], m3.shape[-1], r3.shape[-1]
    x3 = torch.empty_like(r3)
    need = int(lib.frob_solve_workspace_bytes(op, n, nrhs, batch, PREC[prec]))
    ws = torch.empty(need + 256, dtype=torch.uint8, device=m3.device)
    pad = (-ws.data_ptr()) % 256
    info = torch.zeros((batch, 32), dtype=torch.uint8, device=m3.device)
    st = getattr(lib, name)(n, nrhs, batch, m3.data_ptr(), m3.stride(1), m3.stride(0), r3.data_ptr(), r3.stride(1),
                            r3.stride(0), x3.data_ptr(), x3.stride(1), x3.stride(0), PREC[prec], ws.data_ptr() + pad,
                            ws.numel() - pad, info.data_ptr(), torch.cuda.current_stream(m3.device).cuda_stream)
    if st != FROB_OK:
        raise FrobError(f"{name}: {status_str(st)}", st)
    x = x3
    if r.dim() != rhs.dim():
        x = x.squeeze(-1)
    if m.dim() == 2:
        x = x[0]
    res = Result(x, info)
    if check:
        check_info(res.info(), name)
    if on_host:
        res.x = res.x.cpu()
    return res


def frob_solve(m: torch.Tensor, rhs: torch.Tensor, prec: str = "fp64", check: bool = True) -> Result:
    """Solve M X = RHS by Frobenius inversion without forming M^{-1} (Sec. 3);
    m: (n, n) or (batch, n, n); rhs: (..., n) or (..., n, nrhs)."""
    return _solve("frob_solve", 0, m, rhs, prec, check)


def cplx_lu_solve(m: torch.Tensor, rhs: torch.Tensor, prec: str = "fp64", check: bool = True) -> Result:
    """Solve M X = RHS by complex LU with partial pivoting (baseline)."""
    return _solve("cplx_lu_solve", 1, m, rhs, prec, check)


ROUTE = {"frob": 0, "cplx_lu": 1}


class NewtonResult:
    """Output of a Newton driver: the result tensor(s), the per-matrix step
    counts and the device-side info records."""

    def __init__(self, out, steps: torch.Tensor, info: torch.Tensor):
        self.out = out
        self.steps_dev = steps
        self.info_dev = info

    def steps(self) -> np.ndarray:
        return self.steps_dev.cpu().numpy()

    def info(self) -> np.ndarray:
        return parse_info(self.info_dev)


def _batch3(t: torch.Tensor, what: str, prec: str) -> torch.Tensor:
    if t.dtype != _cdtype(prec) or not t.is_cuda:
        raise TypeError(f"{what}: expected a CUDA {_cdtype(prec)} tensor for prec={prec}")
    t3 = t.unsqueeze(0) if t.dim() == 2 else t
    if t3.dim() != 3:
        raise ValueError(f"{what}: expected 2 or 3 dimensions, got {tuple(t.shape)}")
    return t3 if t3.stride(-1) == 1 else t3.contiguous()


def _ws(need: int, dev) -> tuple:
    ws = torch.empty(need + 256, dtype=torch.uint8, device=dev)
    pad = (-ws.data_ptr()) % 256
    return ws, ws.data_ptr() + pad, ws.numel() - pad


def _newton_call(kind: int, m: torch.Tensor, prec: str, route: str, eps: float, kmax: int, check: bool, what: str,
                 ns_tol: float = 1e-14) -> NewtonResult:
    lib = load()
    m3 = _batch3(m, what, prec)
    batch, n = m3.shape[0], m3.shape[-1]
    if m3.shape[-2] != n:
        raise ValueError(f"{what}: expected square matrices")
    x3 = torch.empty((batch, n, n), dtype=m3.dtype, device=m3.device)
    need = int(lib.frob_newton_workspace_bytes(n, batch, PREC[prec], ROUTE[route]))
    if need == 0:
        raise FrobError(f"{what}: unsupported precision / route", FROB_ERR_UNSUPPORTED)
    ws, wp, wb = _ws(need, m3.device)
    info = torch.zeros((batch, 32), dtype=torch.uint8, device=m3.device)
    steps = torch.zeros(batch, dtype=torch.int32, device=m3.device)
    o = _opts(prec, ns_tol=ns_tol)
    with torch.cuda.device(m3.device):
        st = lib.frob_newton(kind, ROUTE[route], n, batch, m3.data_ptr(), m3.stride(1), m3.stride(0), x3.data_ptr(),
                             x3.stride(1), x3.stride(0), ctypes.byref(o), float(eps), int(kmax), wp, wb,
                             info.data_ptr(), steps.data_ptr(), torch.cuda.current_stream(m3.device).cuda_stream)
    if st != FROB_OK:
        raise FrobError(f"{what}: {status_str(st)}", st)
    res = NewtonResult(x3 if m.dim() == 3 else x3[0], steps, info)
    if check:
        check_info(res.info(), what)
    return res


def sign(m: torch.Tensor, prec: str = "fp64", route: str = "frob", eps: float = 1e-3, kmax: int = 100,
         check: bool = True) -> NewtonResult:
    """Matrix sign function by Newton's iteration X <- (X + X^{-1})/2 with
    the stopping rule of Sec. 5.3 (relative change in the max norm <= eps,
    at most kmax steps); every inverse a Frobenius inversion (route "frob")
    or, as the baseline, a complex-LU inversion (route "cplx_lu")."""
    return _newton_call(0, m, prec, route, eps, kmax, check, "sign")


def polar(x: torch.Tensor, prec: str = "fp64", route: str = "frob", eps: float = 1e-3, kmax: int = 100,
          check: bool = True) -> NewtonResult:
    """Polar decomposition X = Q P (Sec. 5.5): Q by X <- (X + X^{-H})/2 with
    the stopping rule of Sec. 5.3, P = Q^H X.  ``out`` is (Q, P)."""
    lib = load()
    x3 = _batch3(x, "polar", prec)
    batch, n = x3.shape[0], x3.shape[-1]
    q3 = torch.empty((batch, n, n), dtype=x3.dtype, device=x3.device)
    p3 = torch.empty_like(q3)
    need = int(lib.frob_polar_workspace_bytes(n, batch, PREC[prec], ROUTE[route]))
    if need == 0:
        raise FrobError("polar: unsupported precision / route", FROB_ERR_UNSUPPORTED)
    ws, wp, wb = _ws(need, x3.device)
    info = torch.zeros((batch, 32), dtype=torch.uint8, device=x3.device)
    steps = torch.zeros(batch, dtype=torch.int32, device=x3.device)
    o = _opts(prec)
    with torch.cuda.device(x3.device):
        st = lib.frob_polar(ROUTE[route], n, batch, x3.data_ptr(), x3.stride(1), x3.stride(0), q3.data_ptr(),
                            q3.stride(1), q3.stride(0), p3.data_ptr(), p3.stride(1), p3.stride(0), ctypes.byref(o),
                            float(eps), int(kmax), wp, wb, info.data_ptr(), steps.data_ptr(),
                            torch.cuda.current_stream(x3.device).cuda_stream)
    if st != FROB_OK:
        raise FrobError(f"polar: {status_str(st)}", st)
    out = (q3, p3) if x.dim() == 3 else (q3[0], p3[0])
    res = NewtonResult(out, steps, info)
    if check:
        check_info(res.info(), "polar")
    return res


def sylvester(a: torch.Tensor, b: torch.Tensor | None, c: torch.Tensor, prec: str = "fp64", route: str = "frob",
              eps: float = 1e-1, kmax: int = 100, lyapunov: bool = False, check: bool = True) -> NewtonResult:
    """Y with A Y + Y B = C (Sec. 5.4) from the sign of [[A, -C], [0, -B]];
    ``lyapunov=True`` takes B = A^H (b is ignored).  ``out`` is Y."""
    lib = load()
    a3 = _batch3(a, "sylvester", prec)
    c3 = _batch3(c, "sylvester", prec)
    batch, p, q = a3.shape[0], a3.shape[-1], c3.shape[-1]
    if lyapunov:
        b3 = a3
    else:
        b3 = _batch3(b, "sylvester", prec)
    if c3.shape[0] != batch or c3.shape[-2] != p or b3.shape[-1] != q:
        raise ValueError("sylvester: A (p, p), B (q, q), C (p, q)")
    y3 = torch.empty((batch, p, q), dtype=a3.dtype, device=a3.device)
    need = int(lib.frob_sylvester_workspace_bytes(p, q, batch, PREC[prec], ROUTE[route]))
    if need == 0:
        raise FrobError("sylvester: unsupported precision / route", FROB_ERR_UNSUPPORTED)
    ws, wp, wb = _ws(need, a3.device)
    info = torch.zeros((batch, 32), dtype=torch.uint8, device=a3.device)
    steps = torch.zeros(batch, dtype=torch.int32, device=a3.device)
    o = _opts(prec)
    with torch.cuda.device(a3.device):
        st = lib.frob_sylvester(ROUTE[route], p, q, batch, a3.data_ptr(), a3.stride(1), a3.stride(0), b3.data_ptr(),
                                b3.stride(1), b3.stride(0), 1 if lyapunov else 0, c3.data_ptr(), c3.stride(1),
                                c3.stride(0), y3.data_ptr(), y3.stride(1), y3.stride(0), ctypes.byref(o), float(eps),
                                int(kmax), wp, wb, info.data_ptr(), steps.data_ptr(),
                                torch.cuda.current_stream(a3.device).cuda_stream)
    if st != FROB_OK:
        raise FrobError(f"sylvester: {status_str(st)}", st)
    res = NewtonResult(y3 if a.dim() == 3 else y3[0], steps, info)
    if check:
        check_info(res.info(), "sylvester")
    return res


def frob_inv_bicomplex(a: torch.Tensor, b: torch.Tensor, prec: str = "fp64", check: bool = True,
                       ns_tol: float = 1e-14):
    """(A + jB)^{-1} = Y0 + jY1 for bicomplex matrices (j^2 = -1, j commuting
    with i; the m = 2 iterated quadratic extension of Sec. 2.4): Frobenius
    inversion over C with complex inversions by frob_inv and complex products
    by Gauss multiplication.  Returns (Y0, Y1, info)."""
    lib = load()
    a3 = _batch3(a, "frob_inv_bicomplex", prec if prec in ("fp32", "fp64") else "fp64")
    b3 = _batch3(b, "frob_inv_bicomplex", prec if prec in ("fp32", "fp64") else "fp64")
    batch, n = a3.shape[0], a3.shape[-1]
    if a3.shape != b3.shape or a3.shape[-2] != n:
        raise ValueError("frob_inv_bicomplex: A and B must be (n, n) or (batch, n, n) of the same shape")
    y0 = torch.empty((batch, n, n), dtype=a3.dtype, device=a3.device)
    y1 = torch.empty_like(y0)
    need = int(lib.frob_inv_bicomplex_workspace_bytes(n, batch, PREC[prec]))
    if need == 0:
        raise FrobError("frob_inv_bicomplex: unsupported precision", FROB_ERR_UNSUPPORTED)
    ws, wp, wb = _ws(need, a3.device)
    info = torch.zeros((batch, 32), dtype=torch.uint8, device=a3.device)
    o = _opts(prec, ns_tol=ns_tol)
    with torch.cuda.device(a3.device):
        st = lib.frob_inv_bicomplex(n, batch, a3.data_ptr(), a3.stride(1), a3.stride(0), b3.data_ptr(), b3.stride(1),
                                    b3.stride(0), y0.data_ptr(), y0.stride(1), y0.stride(0), y1.data_ptr(),
                                    y1.stride(1), y1.stride(0), ctypes.byref(o), wp, wb, info.data_ptr(),
                                    torch.cuda.current_stream(a3.device).cuda_stream)
    if st != FROB_OK:
        raise FrobError(f"frob_inv_bicomplex: {status_str(st)}", st)
    if check:
        check_info(parse_info(info), "frob_inv_bicomplex")
    if a.dim() == 2:
        return y0[0], y1[0], info
    return y0, y1, info


def aug_real_solve(m: torch.Tensor, rhs: torch.Tensor, prec: str = "fp64", check: bool = True) -> Result:
    """Solve M X = RHS through the 2n real augmented system [[A, -B], [B, A]]
    by real LU (the third method of Sec. 5.2, a comparator)."""
    return _solve("aug_real_solve", 2, m, rhs, prec, check)


def inv_adjoint(x: torch.Tensor, g: torch.Tensor, prec: str | None = None) -> torch.Tensor:
    """grad_M = -X^H G X^H for X = M^{-1} and the gradient G of a real loss
    with respect to X (the library's frob_inv_adjoint kernel)."""
    lib = load()
    if prec is None:
        prec = "fp32" if x.dtype == torch.complex64 else "fp64"
    if x.dtype != _cdtype(prec) or g.dtype != x.dtype or not x.is_cuda:
        raise TypeError("inv_adjoint: X and G must be CUDA tensors of the same complex dtype")
    x3 = (x if x.dim() == 3 else x.unsqueeze(0))
    g3 = (g if g.dim() == 3 else g.unsqueeze(0))
    if x3.stride(-1) != 1:
        x3 = x3.contiguous()
    if g3.stride(-1) != 1:
        g3 = g3.contiguous()
    batch, n = x3.shape[0], x3.shape[-1]
    out = torch.empty((batch, n, n), dtype=x3.dtype, device=x3.device)
    need = int(lib.frob_workspace_bytes(OP["frob_inv_adjoint"], n, batch, PREC[prec]))
    ws = torch.empty(need + 256, dtype=torch.uint8, device=x3.device)
    pad = (-ws.data_ptr()) % 256
    st = lib.frob_inv_adjoint(n, batch, x3.data_ptr(), x3.stride(1), x3.stride(0), g3.data_ptr(), g3.stride(1),
                              g3.stride(0), out.data_ptr(), out.stride(1), out.stride(0), PREC[prec],
                              ws.data_ptr() + pad, ws.numel() - pad, torch.cuda.current_stream(x3.device).cuda_stream)
    if st != FROB_OK:
        raise FrobError(f"inv_adjoint: {status_str(st)}", st)
    return out if x.dim() == 3 else out[0]


def gemm_tc(a: torch.Tensor, b: torch.Tensor, kind: str = "bf16", out: torch.Tensor | None = None,
            ws: torch.Tensor | None = None) -> torch.Tensor:
    """C = A B^T on the tensor cores (tcgen05): A (batch, M, K), B (batch, N, K)
    FP32 on the GPU, rounded to BF16 or TF32 (round to nearest), FP32
    accumulation.  Returns C (batch, M, N) FP32."""
    lib = load()
    k = {"bf16": 0, "tf32": 1}[kind]
    a3 = a if a.dim() == 3 else a.unsqueeze(0)
    b3 = b if b.dim() == 3 else b.unsqueeze(0)
    if a3.dtype != torch.float32 or b3.dtype != torch.float32 or not a3.is_cuda:
        raise TypeError("gemm_tc: FP32 CUDA tensors expected")
    batch, M, K = a3.shape
    N = b3.shape[1]
    if a3.stride(-1) != 1:
        a3 = a3.contiguous()
    if b3.stride(-1) != 1:
        b3 = b3.contiguous()
    c3 = torch.empty((batch, M, N), dtype=torch.float32, device=a3.device) if out is None else out
    need = int(lib.frob_gemm_tc_workspace_bytes(k, M, N, K, batch))
    if ws is None:
        ws = torch.empty(need + 256, dtype=torch.uint8, device=a3.device)
    pad = (-ws.data_ptr()) % 256
    err = torch.zeros(1, dtype=torch.int32, device=a3.device)
    st = lib.frob_gemm_tc(k, M, N, K, batch, a3.data_ptr(), a3.stride(1), a3.stride(0), b3.data_ptr(), b3.stride(1),
                          b3.stride(0), c3.data_ptr(), c3.stride(1), c3.stride(0), ws.data_ptr() + pad,
                          ws.numel() - pad, err.data_ptr(), torch.cuda.current_stream(a3.device).cuda_stream)
    if st != FROB_OK:
        raise FrobError(f"gemm_tc: {status_str(st)}", st)
    e = int(err.item())
    if e != 0:
        raise FrobError(f"gemm_tc: device status {status_str(e)}", e)
    return c3 if (a.dim() == 3 or out is not None) else c3[0]


def gemm_f64(a: torch.Tensor, b: torch.Tensor, trans_a: bool = False, trans_b: bool = False,
             alpha: float = 1.0, beta: float = 0.0, out: torch.Tensor | None = None,
             ws: torch.Tensor | None = None) -> torch.Tensor:
    """C = alpha op(A) op(B) + beta C in FP64 as exact BF16 digit products on
    the tensor cores: A (batch, M, K) (or (batch, K, M) with trans_a), B
    (batch, K, N) (or (batch, N, K) with trans_b), FP64 on the GPU, M and
    N >= 128.  Returns C (batch, M, N) FP64 (the `out` tensor when given)."""
    lib = load()
    a3 = a if a.dim() == 3 else a.unsqueeze(0)
    b3 = b if b.dim() == 3 else b.unsqueeze(0)
    if a3.dtype != torch.float64 or b3.dtype != torch.float64 or not a3.is_cuda:
        raise TypeError("gemm_f64: FP64 CUDA tensors expected")
    if a3.stride(-1) != 1:
        a3 = a3.contiguous()
    if b3.stride(-1) != 1:
        b3 = b3.contiguous()
    batch = a3.shape[0]
    M, K = (a3.shape[2], a3.shape[1]) if trans_a else (a3.shape[1], a3.shape[2])
    N = b3.shape[1] if trans_b else b3.shape[2]
    if (b3.shape[2] if trans_b else b3.shape[1]) != K or b3.shape[0] != batch:
        raise ValueError("gemm_f64: inner dimensions or batch differ")
    if out is None:
        c3 = torch.empty((batch, M, N), dtype=torch.float64, device=a3.device)
        beta = 0.0
    else:
        c3 = out if out.dim() == 3 else out.unsqueeze(0)
        if c3.stride(-1) != 1 or tuple(c3.shape) != (batch, M, N) or c3.dtype != torch.float64:
            raise ValueError("gemm_f64: out must be a row-major FP64 (batch, M, N) tensor")
    need = int(lib.frob_gemm_f64_workspace_bytes(M, N, K, batch))
    if need == 0:
        raise ValueError("gemm_f64: M and N must be at least 128")
    if ws is None:
        ws = torch.empty(need + 256, dtype=torch.uint8, device=a3.device)
    pad = (-ws.data_ptr()) % 256
    err = torch.zeros(1, dtype=torch.int32, device=a3.device)
    def ld(t):  # a single row's stride is arbitrary (NumPy, torch): any value >= its length serves
        return t.stride(1) if t.shape[1] > 1 else t.shape[2]

    bs_c = c3.stride(0) if batch > 1 else M * ld(c3)
    st = lib.frob_gemm_f64(M, N, K, batch, a3.data_ptr(), ld(a3), a3.stride(0), int(trans_a),
                           b3.data_ptr(), ld(b3), b3.stride(0), int(trans_b), c3.data_ptr(), ld(c3),
                           bs_c, float(alpha), float(beta), ws.data_ptr() + pad, ws.numel() - pad, err.data_ptr(),
                           torch.cuda.current_stream(a3.device).cuda_stream)
    if st != FROB_OK:
        raise FrobError(f"gemm_f64: {status_str(st)}", st)
    e = int(err.item())
    if e != 0:
        raise FrobError(f"gemm_f64: device status {status_str(e)}", e)
    if out is not None:
        return out
    return c3 if a.dim() == 3 else c3[0]


def draw_mu(seed: int, b: int, attempt: int = 0) -> float:
    """Host copy of the library's SplitMix64 draw of mu (for reporting only;
    the kernels draw mu themselves)."""
    mask = (1 << 64) - 1
    ctr = ((b & 0xFFFFFFFF) << 32) + (attempt & 0xFFFFFFFF) + 1
    z = (seed + ctr * 0x9E3779B97F4A7C15) & mask
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & mask
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & mask
    z ^= z >> 31
    return ((z >> 11) + 0.5) * 2.0 ** -53
