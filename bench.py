"""Benchmark: Frobenius inversion of Hermitian positive definite matrices on
one GB300, against the complex-Cholesky baseline on the same GPU.

Workload: batch 64 of complex FP64 n = 512 HPD matrices M = Q diag(lam) Q^H,
Q from the QR of a complex Gaussian matrix, lam log-uniform on [1, 1e4]
(seeded, synthetic).  One step = one frob_inv_hpd call over the whole batch
(split, two Cholesky factorisations, four triangular solves, the symmetric
product, the final product and the interleaved output; Sec. 4.3).

Metric: complex inversions per second (whole job), with TFLOP/s (executed and
nominal 8 n^3) and the relative residual reported beside it.  The input batch
(268 MB) is larger than L2 (129 MB), so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs its own batch (weak scaling) and rank
0 prints one JSON line with the whole-job throughput.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_ORDER = 512
BATCH = 64
SEED = 2
WORKLOAD = "hpd_batch64_n512_fp64"
METRIC = "complex inversions/s (Frobenius-Cholesky vs complex Cholesky), 1 GB300, equal residual"
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12  # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz = 1.259 TFLOP/s
# DRAM bytes (read + write) of one launch of the final product with the
# interleaving epilogue (32 matrices of order 512), from one ncu capture of
# the current kernel: profiles/gemm_frobout_f64_hpd_b64_n512.md
TRAFFIC_PER_LAUNCH = {"gemm<f64,op0,op0,frob_out>": 226.1e6}


def algorithmic_flops(n, batch):
    """Real flops each kernel family of frob_inv_hpd must do per call (Sec. 4.3,
    Algorithm "Frobenius inversion with Cholesky decomposition")."""
    n3 = float(n) ** 3 * batch
    return {
        "trsm<f64,op1,upper>": n3,                # R1 X2 = X1, n right-hand sides
        "gemm<f64,op0,op0,frob_out>": 2 * n3,     # X7 = X2 X6 (+ interleaved output)
        "trsm<f64,op0,lower>": n3,                # R1^T X1 = B
        "gemm<f64,op1,op0,axpby>": 4 * n3 / 3,    # S = A - X1^T X1 and X6 = X5^T X5 (k >= max(i, j)), lower tiles
        "gemm<f64,op0,op0,axpby>": n3 / 3,        # X5 = L2^{-1}, recursive triangular inverse (joined pairs)
        "gemm<f64,op0,op2,axpby>": 2 * n3 / 3,    # trailing updates of the two Cholesky factorisations
    }


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _gen_inputs(n, batch, seed):
    from paper_2208_01239_gb300 import workloads as W
    return W.hpd(n, batch=batch, seed=seed, return_parts=True)


def _clock_sampler():
    try:
        return subprocess.Popen(
            ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
             "--format=csv,noheader,nounits", "-lms", "200"],
            stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_summary(proc, gpu_index):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, smax, reasons = [], None, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9 or f[0] != str(gpu_index):
            continue
        try:
            sm.append(float(f[1]))
            smax = float(f[2])
        except ValueError:
            continue
        for name, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
            "samples": len(sm)}


def run_reference(args):
    """The CPU oracle (plain C FP64, Frobenius inversion with Cholesky,
    Sec. 4.3) timed as it stands on the host cores, on a bounded sample of the
    same workload per step."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    sample = 2
    ms, _, _ = _gen_inputs(N_ORDER, sample, SEED)
    oracle.build()
    for _ in range(args.warmup):
        for b in range(sample):
            oracle.frob_inv_chol(ms[b])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for b in range(sample):
            oracle.frob_inv_chol(ms[b])
    dt = time.perf_counter() - t0
    value = sample * args.steps / dt
    cores = oracle.num_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "inversions/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_ORDER, "batch": BATCH, "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "inversions/s", "cores": cores, "kind": "oracle",
                         "sample": f"{sample} of the {BATCH} n={N_ORDER} HPD matrices per step, "
                                   "oracle frob_inv_chol (plain C FP64, OpenMP)"},
        "e2e": {"value": value, "unit": "inversions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def residual_fro(m, x):
    """||M X - I||_F / (||M||_F ||X||_F) in FP64 (numpy)."""
    import numpy as np
    r = m @ x - np.eye(m.shape[0])
    return float(np.linalg.norm(r) / (np.linalg.norm(m) * np.linalg.norm(x)))


def cpu_baseline(ms, budget_s=12.0):
    """Oracle (plain C FP64 Frobenius-Cholesky) on a bounded sample."""
    import oracle
    oracle.build()
    oracle.frob_inv_chol(ms[0])
    done, t0 = 0, time.perf_counter()
    while done < len(ms) and time.perf_counter() - t0 < budget_s:
        oracle.frob_inv_chol(ms[done])
        done += 1
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": "inversions/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{done} of the {len(ms)} n={N_ORDER} HPD matrices, oracle frob_inv_chol (plain C FP64, "
                      f"OpenMP), {dt:.1f} s"}


def measure_batched(frob, dev, steps, rank):
    """1024 matrices with n uniform in [32, 512], A, B iid N(0, 1): the mixed
    Frobenius form and the FP64 complex-LU baseline, both through
    frob_inv_batched (one call per step, a fixed launch sequence), timed as
    CUDA-graph replays of the call (and eagerly, for reference)."""
    import numpy as np
    import torch
    from paper_2208_01239_gb300 import workloads as W
    sizes, mats = W.uneven_batch(1024, 32, 512, seed=4 + 1000 * rank)
    out = {"workload": "uneven_1024_n32-512_c128", "sum_n3": float(np.sum(np.asarray(sizes, dtype=np.float64) ** 3))}
    for name, op, prec in (("frob_inv mixed_bf16", "frob_inv", "mixed_bf16"), ("cplx_lu_inv fp64", "cplx_lu_inv", "fp64")):
        plan = frob.Batched(sizes, op=op, prec=prec, device=dev)
        for dst, m in zip(plan.inputs, mats):
            dst.copy_(torch.from_numpy(m))
        plan.run()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            plan.run()
        e1.record()
        torch.cuda.synchronize(dev)
        ms_eager = e0.elapsed_time(e1) / steps
        # the same call captured once in a CUDA graph and replayed (the fixed
        # launch sequence of frob_inv_batched is capture-safe)
        side = torch.cuda.Stream(dev)
        side.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(side):
            plan.run()
        torch.cuda.current_stream(dev).wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            plan.run()
        graph.replay()
        torch.cuda.synchronize(dev)
        e0.record()
        for _ in range(steps):
            graph.replay()
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / steps
        inf = plan.info()
        worst = 0.0
        for k in range(0, 1024, 128):
            m = torch.from_numpy(mats[k]).to(dev)
            x = plan.outputs[k]
            r = m @ x - torch.eye(m.shape[0], dtype=m.dtype, device=dev)
            worst = max(worst, (torch.linalg.norm(r) / (torch.linalg.norm(m) * torch.linalg.norm(x))).item())
        out[name] = {"ms_per_step": ms, "inversions_per_s": 1024 / (ms * 1e-3), "timing": "CUDA graph replay",
                     "ms_per_step_eager": ms_eager, "inversions_per_s_eager": 1024 / (ms_eager * 1e-3),
                     "status_ok": int((inf["status"] == 0).sum()), "residual_fro_max_sampled": worst}
        del graph
        del plan
    a, b = out["frob_inv mixed_bf16"], out["cplx_lu_inv fp64"]
    out["speedup_vs_cplx_lu"] = b["ms_per_step"] / a["ms_per_step"]
    return out


def measure_newton(frob, dev):
    """The Newton drivers at the smallest sizes of the paper's experiments
    (Sec. 5.3-5.5), FP64, with its stopping rules: the matrix sign of
    X = Z J Z^{-1} (n = 2100, eps = 1e-3), the polar decomposition of X = U P
    (n = 2100, eps = 1e-3) and the Sylvester equation with p = q = 1050
    (eps = 1e-1); every inverse a Frobenius inversion or, as the baseline,
    a complex-LU inversion.  Wall time of one driver call (CUDA events; the
    driver reads a 4-byte count from the device after each step), steps, and
    the relative forward error (max norm) against the answer the
    construction fixes."""
    import numpy as np
    import torch
    from paper_2208_01239_gb300 import workloads as W

    def rel(a, b):
        return float(np.abs(a - b).max() / np.abs(b).max())

    def timed_call(f):
        f()  # warm-up (workspace, first-use setup)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        r = f()
        e1.record()
        torch.cuda.synchronize(dev)
        return r, e0.elapsed_time(e1)

    out = {}
    n = 2100
    x, s = W.sign_case(n, seed=61)
    dx = torch.from_numpy(x).to(dev)
    res = {}
    for route in ("frob", "cplx_lu"):
        r, ms = timed_call(lambda: frob.sign(dx, route=route, eps=1e-3, kmax=100, check=False))
        k = int(r.steps()[0])
        res[route] = {"ms": ms, "steps": k, "ms_per_step": ms / max(k, 1),
                      "forward_error": rel(r.out.cpu().numpy(), s)}
    out["sign_n2100"] = res
    x, u, pm = W.polar_case(n, seed=62)
    dx = torch.from_numpy(x).to(dev)
    res = {}
    for route in ("frob", "cplx_lu"):
        r, ms = timed_call(lambda: frob.polar(dx, route=route, eps=1e-3, kmax=100, check=False))
        k = int(r.steps()[0])
        q, p_ = (t.cpu().numpy() for t in r.out)
        res[route] = {"ms": ms, "steps": k, "ms_per_step": ms / max(k, 1), "forward_error_q": rel(q, u),
                      "forward_error_p": rel(p_, pm)}
    out["polar_n2100"] = res
    a, b, c, y = W.sylvester_case(1050, 1050, seed=63)
    da, db, dc = (torch.from_numpy(t).to(dev) for t in (a, b, c))
    res = {}
    for route in ("frob", "cplx_lu"):
        r, ms = timed_call(lambda: frob.sylvester(da, db, dc, route=route, eps=1e-1, kmax=100, check=False))
        k = int(r.steps()[0])
        res[route] = {"ms": ms, "steps": k, "ms_per_step": ms / max(k, 1),
                      "forward_error": rel(r.out.cpu().numpy(), y)}
    out["sylvester_p1050_q1050"] = res
    return out


def measure_accuracy(frob, dev):
    """The accuracy experiments of Sec. 5.1, 5.2 and 5.6 at kappa = 10, FP64:
    left and right relative residuals in the paper's max norm (eq. "backerr":
    ||Y X - I||_max / (||X||_max ||Y||_max), ||A + iB||_max = max(max|a_ij|,
    max|b_ij|)) of Frobenius inversion against complex LU (general matrices,
    the kappa-controlled generator) and against complex Cholesky (HPD,
    kappa(X) = 10); and relative forward errors of linear solves (x, y
    uniform on [-1, 1], c + id = M (x + iy)) by Frobenius, complex LU and
    the 2n real augmented system.  Residuals computed on the host in FP64."""
    import numpy as np
    import torch
    from paper_2208_01239_gb300 import workloads as W

    def mx(a):
        return max(float(np.abs(a.real).max()), float(np.abs(a.imag).max()))

    def res(x, y):
        i = np.eye(x.shape[0])
        return mx(y @ x - i) / (mx(x) * mx(y)), mx(x @ y - i) / (mx(x) * mx(y))

    out = {"kappa": 10.0, "norm": "max of |Re|, |Im| entries (eq. maxnorm)"}
    g = np.random.default_rng(13)
    for n in (64, 512, 2048):
        m = W.kappa_controlled(n, 10.0, seed=80 + n)
        dm = torch.from_numpy(m).to(dev)
        row = {}
        for name, f in (("frob_inv", frob.frob_inv), ("cplx_lu_inv", frob.cplx_lu_inv)):
            y = f(dm, check=False).x.cpu().numpy()
            rl, rr = res(m, y)
            row[name] = {"res_L": rl, "res_R": rr}
        h = W.hpd_kappa(n, 10.0, seed=90 + n)
        dh = torch.from_numpy(h).to(dev)
        for name, f in (("frob_inv_hpd", frob.frob_inv_hpd), ("cplx_chol_inv", frob.cplx_chol_inv)):
            y = f(dh, check=False).x.cpu().numpy()
            rl, rr = res(h, y)
            row[name] = {"res_L": rl, "res_R": rr}
        xt = g.uniform(-1, 1, (n, 1)) + 1j * g.uniform(-1, 1, (n, 1))
        rhs = torch.from_numpy(m @ xt).to(dev)
        for name, f in (("frob_solve", frob.frob_solve), ("cplx_lu_solve", frob.cplx_lu_solve),
                        ("aug_real_solve", frob.aug_real_solve)):
            x = f(dm, rhs, check=False).x.cpu().numpy()
            row[name] = {"forward_error": float(np.abs(x - xt).max() / np.abs(xt).max())}
        out[f"n{n}"] = row
    return out


def measure_config3_fp32(frob, dev):
    """The ill-conditioned construction (A = I, B = Q N Q^T, s = 1 - 1e-6,
    kappa(M) ~ 2e6) in FP32 at n = 512: relative forward error (max norm)
    of Frobenius inversion and of complex LU against the FP64 inverse of the
    FP32-rounded input (LAPACK through numpy on the host), and the residual
    ||M X - I||_F / (||M||_F ||X||_F).  S = (1 - s^2) I ~ 2e-6 I is formed
    by cancellation, which FP32 cannot resolve."""
    import numpy as np
    import torch
    from paper_2208_01239_gb300 import workloads as W
    n = 512
    m, _ = W.ill_conditioned(n, seed=5)
    m32 = m.astype(np.complex64)
    m64 = m32.astype(np.complex128)
    ref = np.linalg.inv(m64)
    out = {"n": n, "kappa": float(np.linalg.cond(m64))}
    for name, f in (("frob_inv", frob.frob_inv), ("cplx_lu_inv", frob.cplx_lu_inv)):
        x = f(torch.from_numpy(m32).to(dev), prec="fp32", check=False).x.cpu().numpy().astype(np.complex128)
        r = m64 @ x - np.eye(n)
        out[name] = {"forward_error": float(np.abs(x - ref).max() / np.abs(ref).max()),
                     "residual_fro": float(np.linalg.norm(r) / (np.linalg.norm(m64) * np.linalg.norm(x)))}
    return out


def measure_solve(frob, dev, steps):
    """Linear systems (Sec. 5.2): 16 systems of order 512, one right-hand
    side, A and B from the kappa = 10 generator of Sec. 5.1 and x, y uniform
    on [-1, 1] with c + id = M (x + iy); and the ill-conditioned construction
    of Sec. 3 (kappa(M) ~ 2e6, kappa(A) = kappa(B) = 1).  Frobenius solve vs
    complex-LU solve: relative forward error (max norm) and solves/s."""
    import numpy as np
    import torch
    from paper_2208_01239_gb300 import workloads as W
    n, batch = 512, 16
    g = np.random.default_rng(12)
    out = {}
    cases = {}
    ms = np.stack([W.kappa_controlled(n, 10.0, seed=100 + k) for k in range(batch)])
    xs = g.uniform(-1, 1, (batch, n, 1)) + 1j * g.uniform(-1, 1, (batch, n, 1))
    cases["kappa10"] = (ms, ms @ xs, xs)
    mi = []
    xi = []
    for k in range(batch):
        m, minv = W.ill_conditioned(n, seed=200 + k)
        b = g.standard_normal((n, 1)) + 1j * g.standard_normal((n, 1))
        mi.append(m)
        xi.append((minv @ b, b))
    cases["ill_conditioned"] = (np.stack(mi), np.stack([b for _, b in xi]), np.stack([x for x, _ in xi]))
    for cname, (m, rhs, xtrue) in cases.items():
        dm = torch.from_numpy(np.ascontiguousarray(m)).to(dev)
        dr = torch.from_numpy(np.ascontiguousarray(rhs)).to(dev)
        res = {}
        for method in ("frob_solve", "cplx_lu_solve"):
            f = getattr(frob, method)
            x = f(dm, dr, check=False).x
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(steps):
                x = f(dm, dr, check=False).x
            e1.record()
            torch.cuda.synchronize(dev)
            ms_ = e0.elapsed_time(e1) / steps
            xn = x.cpu().numpy()
            fe = max(float(np.max(np.abs(np.concatenate([(xn[k] - xtrue[k]).real.ravel(), (xn[k] - xtrue[k]).imag.ravel()])))) /
                     float(max(np.abs(xtrue[k].real).max(), np.abs(xtrue[k].imag).max())) for k in range(batch))
            res[method] = {"forward_error_max": fe, "solves_per_s": batch / (ms_ * 1e-3), "ms_per_step": ms_}
        out[cname] = res
    out["n"] = n
    out["batch"] = batch
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--once", action="store_true",
                    help="run the workload twice (one warm-up call) and exit: the command profiled by ncu")
    ap.add_argument("--once-mixed", action="store_true",
                    help="as --once, for the mixed-precision form")
    ap.add_argument("--no-batched", action="store_true", help="skip the 1024-matrix uneven workload")
    ap.add_argument("--no-newton", action="store_true", help="skip the Newton-driver workloads (sign, polar, Sylvester)")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the kappa = 10 accuracy study")
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="matrices per step for --once / --once-mixed (profiling a smaller case)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2208_01239_gb300 import build as fbuild
    from paper_2208_01239_gb300 import flops
    from paper_2208_01239_gb300 import frob

    world, rank, local = _dist()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    fbuild.build()
    lib = frob.load()

    batch_n = args.batch if (args.once or args.once_mixed) else BATCH
    ms, qs, lams = _gen_inputs(N_ORDER, batch_n, SEED + rank)
    m_host = torch.from_numpy(ms).pin_memory()
    m_dev = m_host.to(dev)
    x_dev = torch.empty_like(m_dev)
    x_host = torch.empty_like(m_host).pin_memory()
    need = frob.workspace_bytes("frob_inv_hpd", N_ORDER, batch_n)
    ws = torch.empty(need + 256, dtype=torch.uint8, device=dev)
    need_c = frob.workspace_bytes("cplx_chol_inv", N_ORDER, batch_n)
    ws_c = torch.empty(need_c + 256, dtype=torch.uint8, device=dev)
    info = torch.zeros((batch_n, 32), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        frob.frob_inv_hpd(m_dev, out=x_dev, ws=ws, info=info, check=False)

    if args.once:
        step()
        step()
        torch.cuda.synchronize(dev)
        frob.check_info(frob.parse_info(info), "frob_inv_hpd")
        return 0
    if args.once_mixed:
        need_m = frob.workspace_bytes("frob_inv_hpd", N_ORDER, batch_n, "mixed_bf16")
        ws_m = torch.empty(need_m + 256, dtype=torch.uint8, device=dev)
        for _ in range(2):
            frob.frob_inv_hpd(m_dev, prec="mixed_bf16", out=x_dev, ws=ws_m, info=info, check=False)
        torch.cuda.synchronize(dev)
        frob.check_info(frob.parse_info(info), "frob_inv_hpd mixed")
        return 0

    def step_baseline():
        frob.cplx_chol_inv(m_dev, out=x_dev, ws=ws_c, info=info, check=False)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)

    def timed(fn, steps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(steps):
            fn()
        ev1.record(stream)
        barrier()
        ms_ = ev0.elapsed_time(ev1)
        if world > 1:
            t = torch.tensor([ms_], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_ = float(t.item())
        return ms_

    # warm-up and correctness of the timed configuration
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    inf = frob.parse_info(info)
    frob.check_info(inf, "frob_inv_hpd")
    x0 = x_dev.cpu().numpy()
    res = max(residual_fro(ms[b], x0[b]) for b in (0, BATCH // 2, BATCH - 1))

    # timed region (device): K steps, clocks sampled meanwhile
    launches0 = lib.frob_kernel_launches()
    clk = _clock_sampler()
    time.sleep(0.3)
    t_ms = timed(step, args.steps)
    clocks = _clock_summary(clk, local)
    launches = lib.frob_kernel_launches() - launches0
    ms_per_step = t_ms / args.steps
    value = world * BATCH / (ms_per_step * 1e-3)
    # per-kernel device times: a separate profiled pass of the same steps, in
    # which the library brackets every launch with CUDA events on its stream
    # and runs batch slices one after the other (so each kernel runs alone)
    prof_steps = min(args.steps, 3)
    frob.profile_enable(True)
    tp_ms = timed(step, prof_steps) / prof_steps
    frob.profile_enable(False)
    prof = {k: (v[0] * args.steps / prof_steps, v[1] * args.steps / prof_steps)
            for k, v in frob.profile_report().items()}

    # baseline on the same GPU (complex Cholesky inversion)
    for _ in range(args.warmup):
        step_baseline()
    tb_ms = timed(step_baseline, args.steps) / args.steps
    torch.cuda.synchronize(dev)
    xb = x_dev.cpu().numpy()
    res_b = max(residual_fro(ms[b], xb[b]) for b in (0, BATCH // 2, BATCH - 1))

    # the mixed form on the same workload: FP32 Cholesky-Frobenius start,
    # Newton-Schulz refinement with FP64-accurate products on the BF16 tensor
    # cores, same residual gate; at the default tolerance (7-digit residuals)
    # and at 1e-15 (8-digit residuals, a residual floor near the FP64 paths')
    need_m = frob.workspace_bytes("frob_inv_hpd", N_ORDER, BATCH, "mixed_bf16")
    ws_m = torch.empty(need_m + 256, dtype=torch.uint8, device=dev)

    def measure_mixed(tol):
        def step_mixed():
            frob.frob_inv_hpd(m_dev, prec="mixed_bf16", out=x_dev, ws=ws_m, info=info, check=False, ns_tol=tol)

        for _ in range(args.warmup):
            step_mixed()
        torch.cuda.synchronize(dev)
        tm_ms = timed(step_mixed, args.steps) / args.steps
        frob.profile_enable(True)
        timed(step_mixed, args.steps)
        frob.profile_enable(False)
        prof_m = frob.profile_report()
        inf_m = frob.parse_info(info)
        xm = x_dev.cpu().numpy()
        res_m = max(residual_fro(ms[b], xm[b]) for b in (0, BATCH // 2, BATCH - 1))
        tot_m = max(sum(v[1] for v in prof_m.values()), 1e-30)
        return {"name": "frob_inv_hpd prec=mixed_bf16", "ns_tol": tol, "value": world * BATCH / (tm_ms * 1e-3),
                "unit": "inversions/s", "ms_per_step": tm_ms, "residual_fro_max_sampled": res_m,
                "residual_fro_max_device": float(inf_m["residual"].max()),
                "status_ok": int((inf_m["status"] == 0).sum()),
                "ns_iters_hist": np.bincount(inf_m["ns_iters"], minlength=1).tolist(),
                "dtype": "bf16 tensor cores + fp32 (results FP64-accurate)",
                "top_kernels": {k: round(v[1] / args.steps, 3) for k, v in
                                sorted(prof_m.items(), key=lambda kv: -kv[1][1])[:6]},
                "top_share": {k: round(v[1] / tot_m, 3) for k, v in
                              sorted(prof_m.items(), key=lambda kv: -kv[1][1])[:6]}}

    mixed = measure_mixed(1e-14)
    mixed_fine = measure_mixed(1e-15)

    batched = None if args.no_batched else measure_batched(frob, dev, max(2, min(args.steps, 3)), rank)
    solve = None if args.no_batched else measure_solve(frob, dev, 3)
    newton = None if (args.no_newton or args.no_batched) else measure_newton(frob, dev)
    accuracy = None if (args.no_accuracy or args.no_batched) else measure_accuracy(frob, dev)
    config3_fp32 = None if (args.no_accuracy or args.no_batched) else measure_config3_fp32(frob, dev)

    # end to end through the public API with host buffers
    def e2e_step():
        m_dev.copy_(m_host, non_blocking=True)
        frob.frob_inv_hpd(m_dev, out=x_dev, ws=ws, info=info, check=False)
        x_host.copy_(x_dev, non_blocking=True)

    for _ in range(2):
        e2e_step()
    te_ms = timed(e2e_step, args.steps) / args.steps
    bytes_io = BATCH * N_ORDER * N_ORDER * 16

    # the dominant kernel family by device time, and its algorithmic rate
    alg = algorithmic_flops(N_ORDER, BATCH)
    top = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    roof = {"bound": "alu", "achieved": None, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": None,
            "traffic": None, "kernel": top,
            "peak_source": "FP64 DFMA pipe: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (derived; measured 1.19)",
            "timing": "CUDA events around each launch on its stream, profiled pass with batch slices serialised",
            "profiled_ms_per_step": tp_ms}
    if top in alg:
        launches_top, ms_top = prof[top]
        ach = alg[top] * args.steps / (ms_top * 1e-3) / 1e12
        roof.update(achieved=ach, frac=ach / FP64_PEAK_TFLOPS, launches_per_step=launches_top / args.steps,
                    flops_per_step=alg[top], ms_per_launch=ms_top / launches_top,
                    traffic=TRAFFIC_PER_LAUNCH.get(top))

    exec_flops = flops.executed("frob_chol", N_ORDER) * BATCH
    tflops_exec = exec_flops / (ms_per_step * 1e-3) / 1e12
    tflops_nom = flops.nominal(N_ORDER) * BATCH / (ms_per_step * 1e-3) / 1e12

    line = {
        "metric": METRIC, "value": value, "unit": "inversions/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_ORDER, "batch": BATCH, "seed": SEED,
                   "lam": "log-uniform [1, 1e4]", "l2": "inputs (268 MB) larger than L2, no flush"},
        "tflops_executed": tflops_exec, "tflops_nominal_8n3": tflops_nom,
        "residual_fro_max_sampled": res,
        "baseline_gpu": {"name": "cplx_chol_inv", "value": world * BATCH / (tb_ms * 1e-3), "unit": "inversions/s",
                         "ms_per_step": tb_ms, "residual_fro_max_sampled": res_b,
                         "tflops_executed": flops.executed("cplx_chol", N_ORDER) * BATCH / (tb_ms * 1e-3) / 1e12},
        "roofline": roof,
        "path_roofline": {"bound": "alu", "achieved": tflops_exec, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                          "frac": tflops_exec / FP64_PEAK_TFLOPS, "what": "whole step, executed FP64 flops"},
        "kernels": {k: {"launches": v[0], "ms_per_step": v[1] / args.steps,
                        "share": v[1] / max(sum(x[1] for x in prof.values()), 1e-30)} for k, v in prof.items()},
        "mixed": mixed,
        "mixed_tol_1e-15": mixed_fine,
        "batched_uneven": batched,
        "linear_solve": solve,
        "newton_drivers": newton,
        "accuracy_kappa10": accuracy,
        "ill_conditioned_fp32": config3_fp32,
        "e2e": {"value": world * BATCH / (te_ms * 1e-3), "unit": "inversions/s", "h2d_bytes_per_step": bytes_io,
                "d2h_bytes_per_step": bytes_io},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(ms)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
