#!/usr/bin/env python
"""Benchmark of the GB300 Iterative Hessian Sketch library.

Metric: IHS time-to-1e-10 relative error (||x - x_OPT||_A / ||x_OPT||_A) of
the mixed-precision form, beside the plain FP64 form, and the SA sketch
kernel's bandwidth against the measured HBM peak.

Workload (default): OLS on a dense 1,048,576 x 500 FP32 matrix with rows
N(0, Sigma), Sigma_ij = 0.5^|i-j|, b = A x* + 0.1 N(0,1), CountSketch
m = 5000 (10 d), seed 0.  A "step" is one whole solve from x = 0 for the
number of iterations the form needs to reach 1e-10 (found once, off the
clock, against x_OPT).  A (2.1 GB) is far larger than L2, so every pass
streams from HBM.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).
"""
import os

for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "IHS time-to-1e-10 rel. error (mixed vs FP64); SA sketch GB/s vs HBM peak"
FALLBACK_HBM = 6800.0
FALLBACK_BF16 = 1900.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def tensor_peak_tf32():
    """Dense TF32 tensor peak: the measured BF16 burst figure times the
    nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s), else the fallback."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 burst x 1.1/2.25"
    return FALLBACK_BF16 * 1.1 / 2.25, "fallback bf16 x 1.1/2.25"


# ---------------------------------------------------------------- clocks ---
class Clocks:
    """nvidia-smi samples (every 50 ms) while the timed region runs."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": len(self.rows)}
        if not self.rows:
            return out
        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [num(r[0]) for r in self.rows if num(r[0])]
        out["sm_mhz"] = statistics.median(sm) if sm else None
        out["sm_max_mhz"] = max((num(r[1]) or 0) for r in self.rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for k, nm in enumerate(names):
            if any(r[3 + k].lower() == "active" for r in self.rows):
                out["reasons"].append(nm)
        return out


# ------------------------------------------------------------ CPU oracle ---
def host_cpu():
    """(threads available, CPU model name) of this host, for the CPU baseline."""
    cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return cores, model


def oracle_time_to_tol(w, n_sample, T, seed=0, iters=3, threads=1, budget_s=None):
    """The FP64 CPU oracle, timed on a bounded sample of the workload: IHS
    iterations (sketch draw, SA, gradient, Gram, Cholesky step) on the first
    n_sample rows (all n by default), on `threads` host threads (the
    multi-core build of the same C loops, bit-identical results).  It runs
    `iters` iterations, or, with budget_s, as many of the T iterations as the
    first one says fit in budget_s (all T: a measured whole solve).  O(n)
    passes are scaled to the full n when sampled; the mean iteration times T
    is the time to 1e-10.  Returns (ms, description, seconds spent, threads,
    iterations run)."""
    import oracle as O
    used = O.use_threads(threads)
    try:
        n = w["n"]
        n_sample = min(n_sample or n, w["A"].shape[0])
        if w.get("A64") is not None and w["A64"].shape[0] == n_sample:
            A = w["A64"]  # promoted once by the caller
        else:
            A = np.ascontiguousarray(w["A"][:n_sample], dtype=np.float64)
        b = np.ascontiguousarray(w["b"][:n_sample])
        m, s = w["m"], w["s"]
        x = np.zeros(A.shape[1])
        t_n = t_g = 0.0
        it, todo = 0, iters
        while it < todo:
            t0 = time.perf_counter()
            bucket, sign = O.hash_draw(seed, it, s, m, n_sample)
            SA = O.sketch(A, m, s, bucket, sign)
            g = O.resid_grad(A, b, x)
            t1 = time.perf_counter()
            H = O.gram(SA, 1.0 / s)
            x = x + O.chol_solve(H, g)
            t2 = time.perf_counter()
            t_n += t1 - t0
            t_g += t2 - t1
            it += 1
            if budget_s is not None and it == 1:
                todo = int(max(1, min(T, budget_s // max(t2 - t0, 1e-9))))
    finally:
        O.use_threads(1)
    per_iter = (t_n * (n / n_sample) + t_g) / it
    core = "%d thread%s" % (used, "" if used == 1 else "s")
    if it == T and n_sample == n:
        desc = ("the whole solve: all %d iterations on the whole %d-row workload, %s"
                % (T, n, core))
    elif n_sample == n:
        desc = ("%d oracle iteration%s on the whole %d-row workload (%s), the mean iteration "
                "times %d iterations" % (it, "" if it == 1 else "s", n, core, T))
    else:
        desc = ("%d oracle iterations on the first %d of %d rows (O(n) passes scaled by %.1f, "
                "m x d Gram whole; %s), the mean iteration times %d iterations"
                % (it, n_sample, n, n / n_sample, core, T))
    return per_iter * T * 1e3, desc, t_n + t_g, used, it


def oracle_iterations_proxy():
    """Iterations the FP64 oracle needs to reach 1e-10 on a proxy of the
    workload with the same m/d = 10 and design (65536 x 100, m = 1000)."""
    import oracle as O
    w = synth.make("ols_dense_ar1", n=65536, d=100, m=1000)
    A = w["A"].astype(np.float64)
    G = A.T @ A
    xo = O.x_opt_ols_normal(A, w["b"])
    xs = O.ihs(A, w["b"], O.OLS, 0.0, 1000, 1, 0, 60)
    for t, x in enumerate(xs):
        if O.err_A(x, xo, G) <= 1e-10:
            return t
    return 60


# ----------------------------------------------------------- GPU harness ---
def x_opt_gpu(A, b):
    """x_OPT off the clock: FP64 normal equations from the FP32 data (exactly
    promoted), Cholesky, three refinement steps with FP64 residuals."""
    import torch
    d = A.shape[1]
    G = torch.zeros((d, d), dtype=torch.float64, device=A.device)
    rhs = torch.zeros(d, dtype=torch.float64, device=A.device)
    CH = 1 << 17
    for i in range(0, A.shape[0], CH):
        Ac = A[i:i + CH].double()
        G += Ac.T @ Ac
        rhs += Ac.T @ b[i:i + CH]
    Lc = torch.linalg.cholesky(G)
    x = torch.cholesky_solve(rhs[:, None], Lc)[:, 0]
    for _ in range(3):
        g = torch.zeros(d, dtype=torch.float64, device=A.device)
        for i in range(0, A.shape[0], CH):
            Ac = A[i:i + CH].double()
            g += Ac.T @ (b[i:i + CH] - Ac @ x)
        x = x + torch.cholesky_solve(g[:, None], Lc)[:, 0]
    return x, G


def max_over_ranks(values, device):
    """Element-wise maximum of a list of floats over the ranks of the default
    process group (the job's time is its slowest rank's); unchanged alone."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(values)
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def err_A(x, xo, G):
    e = x - xo
    return float(((e @ G @ e).clamp_min(0).sqrt() / (xo @ G @ xo).sqrt()).item())


def iterations_to(solver, xo, G, tol, cap=80):
    import torch
    x = torch.zeros(solver.d, dtype=torch.float64, device=xo.device)
    errs = []
    for t in range(cap):
        solver.solve(x, t0=t, iters=1)
        errs.append(err_A(x, xo, G))
        if errs[-1] <= tol:
            return t + 1, errs
    return cap, errs


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("fused.cu", "common.cuh"):  # the fused pass's source and its inline helpers
        h.update(open(os.path.join(ROOT, "paper_1910_14166_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def traffic_for(kernel):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else null)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("kernels", {}).get(kernel)


def run_ours(args, rank, world):
    import torch
    import paper_1910_14166_gb300 as ihs

    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    w = synth.make(args.workload, n=args.n, seed=rank)
    n, d, m, s = w["n"], w["d"], w["m"], w["s"]
    A = torch.from_numpy(w["A"]).cuda()
    b = torch.from_numpy(w["b"]).cuda()
    xo, G = x_opt_gpu(A, b)

    mixed = ihs.IHS(A, b, kind="ols", m=m, s=s, seed=0, precision=args.precision)
    plain = ihs.IHS(A, b, kind="ols", m=m, s=s, seed=0, precision="fp64")
    T_mixed, errs_mixed = iterations_to(mixed, xo, G, 1e-10)
    T_plain, errs_plain = iterations_to(plain, xo, G, 1e-10)

    def solve_steps(solver, T, K):
        x = torch.zeros(d, dtype=torch.float64, device="cuda")
        for _ in range(K):
            x.zero_()
            solver.solve(x, t0=0, iters=T)
        return x

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(solver, T, K, W, profile=False, per_step=None):
        solve_steps(solver, T, W)
        if profile:
            solver.profile(True)
        barrier()
        st = torch.cuda.current_stream()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
        x = torch.zeros(d, dtype=torch.float64, device="cuda")
        ev[0].record(st)
        for k in range(K):  # one event between steps: the per-step times for the median
            x.zero_()
            solver.solve(x, t0=0, iters=T)
            ev[k + 1].record(st)
        barrier()
        ms = ev[0].elapsed_time(ev[K]) / K
        if per_step is not None:
            per_step.extend(ev[k].elapsed_time(ev[k + 1]) for k in range(K))
        prof = solver.profile_read() if profile else None
        if profile:
            solver.profile(False)
        return ms, x, prof

    # setup: ihs_create of the benchmark's context (workspaces from the
    # library's pool, the float-pair copy of b), median of 5 after one
    setup = []
    for it in range(6):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv = ihs.IHS(A, b, kind="ols", m=m, s=s, seed=0, precision=args.precision)
        torch.cuda.synchronize()
        if it:
            setup.append((time.perf_counter() - t0) * 1e3)
        sv.close()
        del sv
    setup_ms = statistics.median(setup)

    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    steps_mixed = []
    ms_mixed, x_m, prof = timed(mixed, T_mixed, args.steps, args.warmup, profile=True,
                                per_step=steps_mixed)
    clk = clocks.stop()
    ms_plain, x_p, prof_plain = timed(plain, T_plain, max(1, args.steps // 2), 1, profile=True)
    err_final = err_A(x_m, xo, G)
    err_final_plain = err_A(x_p, xo, G)

    # max over ranks
    ms_mixed, ms_plain = max_over_ranks([ms_mixed, ms_plain], "cuda")

    # per-kernel roofline from the stage events of the timed region
    hbm, hbm_kind = peaks()
    ms_stage, cnt, launches = prof
    a_bytes = n * d * 4
    fused = cnt["grad"] == 0 and cnt["sketch"] > 0
    lookahead = 0 < cnt["sketch"] < cnt["grad"]
    if fused:
        # one pass: A, the sorted pair list (4 B/row), b as a float pair (8 B/row), SA out
        alg = {"sketch": a_bytes + m * d * 4 + n * 12}
        names = {"sketch": "k_sketch_grad_fused"}
    elif lookahead:
        # look-ahead pipeline: per solve one sketch-only pass, then T fused passes
        # (gradient + SA of the next iteration; the last one without SA)
        alg = {"grad": a_bytes + n * 12 + m * d * 4 * (T_mixed - 1) / T_mixed,
               "sketch": a_bytes + m * d * 4}
        names = {"grad": "k_sketch_grad_fused", "sketch": "k_sketch_dense"}
    else:
        alg = {"sketch": a_bytes + m * d * 4, "grad": a_bytes + n * 8}
        names = {"sketch": "k_sketch_dense", "grad": "k_rg_dense_f32"}
    kernels = {}
    for k in alg:
        avg = ms_stage[k] / max(1, cnt[k])
        gbs = alg[k] / (avg * 1e-3) / 1e9 if avg > 0 else 0.0
        kernels[names[k]] = {"ms_avg": round(avg, 4), "algorithmic_bytes": alg[k],
                             "GB_s": round(gbs, 1), "frac": round(gbs / hbm, 3)}
    # The fused pass is also bound by its FP32 arithmetic: 23 FP32 operations
    # an element (the sketch's FMA, and TwoProd + TwoSum + the low-part FMA for
    # the float-pair residual and again for the gradient), against the FP32
    # peak of 128 operations per clock per SM at the maximum SM clock.
    if "k_sketch_grad_fused" in kernels:
        kf = kernels["k_sketch_grad_fused"]
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = (clk.get("sm_max_mhz") or 2070.0) if isinstance(clk, dict) else 2070.0
        fp32_peak = 128.0 * sms * mhz * 1e6
        ops = 23.0 * n * d
        kf["fp32_ops"] = ops
        kf["fp32_Tops"] = round(ops / (kf["ms_avg"] * 1e-3) / 1e12, 2)
        kf["fp32_peak_Tops"] = round(fp32_peak / 1e12, 2)
        kf["fp32_frac"] = round(ops / (kf["ms_avg"] * 1e-3) / fp32_peak, 3)
    dominant = max(alg, key=lambda k: ms_stage[k])
    kd = kernels[names[dominant]]
    roofline = {"kernel": names[dominant], "bound": "hbm", "achieved": kd["GB_s"], "peak": hbm,
                "unit": "GB/s", "frac": kd["frac"], "peak_kind": hbm_kind,
                "traffic": traffic_for(names[dominant])}
    sk = kernels[names["sketch"]]

    # the mixed form with SA and the gradient in two separate passes, for comparison
    ms_two = None
    if (fused or lookahead) and not args.no_two_pass:
        two = ihs.IHS(A, b, kind="ols", m=m, s=s, seed=0, precision=args.precision, fuse=False)
        ms_two, _, _ = timed(two, T_mixed, max(1, args.steps // 2), 1)
        del two
    # the mixed form with the sketched Hessian factored in FP64 instead of FP32
    ms_f64fac, T_f64fac, errs_f64fac = None, None, None
    if not args.no_two_pass:
        f64f = ihs.IHS(A, b, kind="ols", m=m, s=s, seed=0, precision=args.precision,
                       fp64_factor=True)
        T_f64fac, errs_f64fac = iterations_to(f64f, xo, G, 1e-10)
        ms_f64fac, _, _ = timed(f64f, T_f64fac, max(1, args.steps // 2), 1)
        del f64f

    # the sketch stage as one unit: draw + sort, SA, fix-up of split buckets
    # (the stand-alone sketch kernel, every stage on one stream), and the
    # pipeline's per-iteration sort + fused pass + fix-up from the timed run
    sv = ihs.IHS(A, b, kind="ols", m=m, s=s, seed=0, precision=args.precision, serial=True)
    sv.sketch(0)
    sv.profile(True)
    for t in range(1, 6):
        sv.sketch(t)
    ms_sk, cnt_sk, _ = sv.profile_read()
    sv.close()
    del sv
    sk_parts = {k: ms_sk[k] / max(1, cnt_sk[k]) for k in ("sort", "sketch", "sketch_fix")}
    sk_ms = sum(sk_parts.values())
    sk_bytes = a_bytes + m * d * 4
    sketch_stage = {"what": "sort (draw + counting sort) + SA kernel + fix-up, one stream",
                    "ms": round(sk_ms, 4), **{k + "_ms": round(v, 4) for k, v in sk_parts.items()},
                    "algorithmic_bytes": sk_bytes,
                    "GB_s": round(sk_bytes / (sk_ms * 1e-3) / 1e9, 1),
                    "frac": round(sk_bytes / (sk_ms * 1e-3) / 1e9 / hbm, 3)}
    if lookahead or fused:
        per = {k: ms_stage[k] / max(1, cnt[k]) for k in ("sort", "grad" if lookahead else "sketch",
                                                          "sketch_fix")}
        fb = alg["grad" if lookahead else "sketch"]
        fms = sum(per.values())
        sketch_stage["fused_pipeline"] = {
            "what": "per iteration: sort (on the second stream, overlapped) + fused pass "
                    "(SA of the next iteration and the gradient) + fix-up",
            "ms": round(fms, 4), "algorithmic_bytes": fb,
            "GB_s": round(fb / (fms * 1e-3) / 1e9, 1),
            "frac": round(fb / (fms * 1e-3) / 1e9 / hbm, 3)}

    # the Gaussian comparison sketch (Sec. 2) on the same data: one sketch
    # (G generated in the kernel, SA = G A on the tensor cores) and the solve
    gauss = None
    if not args.no_extra:
        tf32_peak, tf32_kind = tensor_peak_tf32()
        gv = ihs.IHS(A, b, kind="ols", m=m, s=s, seed=0, precision=args.precision,
                     sketch="gaussian", serial=True)
        gv.sketch(0)
        gv.profile(True)
        for t in range(1, 4):
            gv.sketch(t)
        ms_g, cnt_g, _ = gv.profile_read()
        gms = ms_g["sketch"] / max(1, cnt_g["sketch"])
        gflop = 2.0 * m * n * d
        x_g = torch.zeros(d, dtype=torch.float64, device="cuda")
        gv.solve(x_g, iters=2)  # warm-up of the solve path
        gtimes = []
        for _ in range(2):
            x_g.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            gv.solve(x_g, iters=T_mixed)
            e1.record()
            torch.cuda.synchronize()
            gtimes.append(e0.elapsed_time(e1))
        gauss = {"kernel": "k_gauss_tc", "sketch_ms": round(gms, 3),
                 "flops": gflop, "TFLOP_s": round(gflop / (gms * 1e-3) / 1e12, 1),
                 "peak_tf32_TFLOP_s": round(tf32_peak, 1), "peak_kind": tf32_kind,
                 "frac": round(gflop / (gms * 1e-3) / 1e12 / tf32_peak, 3),
                 "solve_ms": round(min(gtimes), 3), "iters": T_mixed,
                 "final_err": err_A(x_g, xo, G)}
        gv.close()
        del gv

    # the large sparse LASSO workload: solve time and the CSC sketch's bandwidth
    c5 = c5_record(ihs, hbm) if not args.no_extra and rank == 0 else None

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        A_h = torch.from_numpy(w["A"]).pin_memory()
        b_h = torch.from_numpy(w["b"]).pin_memory()
        A_d = torch.empty_like(A)
        b_d = torch.empty_like(b)
        del mixed
        st = torch.cuda.current_stream()
        times, copies = [], []
        for it in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            e0, ec, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(st)
            A_d.copy_(A_h, non_blocking=True)
            b_d.copy_(b_h, non_blocking=True)
            ec.record(st)
            sv = ihs.IHS(A_d, b_d, kind="ols", m=m, s=s, seed=0, precision=args.precision)
            x, _ = sv.solve(iters=T_mixed)
            x_host = x.cpu()
            e1.record(st)
            torch.cuda.synchronize()
            sv.close()
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1))
                copies.append(e0.elapsed_time(ec))
        # the host link is shared with the box's other GPU: report the median
        # step and the copy's share of it
        h2d = int(A_h.numel() * 4 + b_h.numel() * 8)
        cp = statistics.median(copies)
        e2e = {"value": round(statistics.median(times), 3), "unit": "ms",
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": int(x_host.numel() * 8),
               "h2d_ms": round(cp, 3), "h2d_GB_s": round(h2d / (cp * 1e-3) / 1e9, 1),
               "steps_ms": [round(t, 2) for t in times]}

    cpu = None
    if rank == 0 and not args.no_cpu:
        cores, model = host_cpu()
        ms_cpu, desc, spent, used, _ = oracle_time_to_tol(w, args.cpu_rows, T_plain,
                                                          threads=cores, budget_s=args.cpu_budget)
        cpu = {"value": round(ms_cpu, 1), "unit": "ms", "cores": used, "kind": "oracle",
               "sample": desc, "cpu_seconds": round(spent, 2), "host_cores": cores,
               "cpu_model": model,
               "build": "the oracle's C loops built with OpenMP: each output summed in the "
                        "serial order, results bit-identical to the one-thread build"}

    res = {
        "metric": METRIC,
        "value": round(ms_mixed, 3),
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_mixed, 3),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": ("f32 A, f64 b and iterate; SA f32 accumulation; Gram %s inputs, f32 "
                  "accumulation; Cholesky factor f32 (the f64 factor of the configuration: "
                  "mixed_fp64_factor_ms); residual and gradient double-float (~48-bit, "
                  "FP64-class)" % args.precision),
        "data": "synthetic",
        "config": config_of(args.workload, n, d, m, s, world),
        "precision": args.precision,
        "iters_to_1e-10": {"mixed": T_mixed, "fp64": T_plain, "mixed_fp64_factor": T_f64fac},
        "final_err": {"mixed": err_final, "fp64": err_final_plain},
        "err_per_iter": {
            "what": "||x^t - x_OPT||_A / ||x_OPT||_A after iteration t = 1, 2, ... (x_OPT by "
                    "FP64 normal equations with refinement)",
            "mixed": [float("%.3g" % e) for e in errs_mixed],
            "mixed_fp64_factor": ([float("%.3g" % e) for e in errs_f64fac]
                                  if errs_f64fac else None),
            "fp64": [float("%.3g" % e) for e in errs_plain]},
        "ms_per_step_median": round(statistics.median(steps_mixed), 3),
        "setup_ms": round(setup_ms, 3),
        "value_with_setup_ms": round(ms_mixed + setup_ms, 3),
        "fp64_time_to_1e-10_ms": round(ms_plain, 3),
        "mixed_speedup_vs_fp64": round(ms_plain / ms_mixed, 3),
        "mixed_two_pass_ms": round(ms_two, 3) if ms_two else None,
        "mixed_fp64_factor_ms": round(ms_f64fac, 3) if ms_f64fac else None,
        "sketch_GB_s": sk["GB_s"],
        "sketch_frac_of_hbm": sk["frac"],
        "sketch_stage": sketch_stage,
        "gaussian_sketch": gauss,
        "lasso_csr_zipf": c5,
        "kernels": kernels,
        "stage_ms_per_iter": {k: round(v / max(1, cnt[k]), 4) for k, v in ms_stage.items()},
        "stage_ms_per_iter_fp64": {k: round(v / max(1, prof_plain[1][k]), 4)
                                   for k, v in prof_plain[0].items()},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    return res


def config_of(workload, n, d, m, s, world):
    """The benchmark's workload, named the same way by both arms."""
    return {"workload": "%s n=%d d=%d m=%d s=%d CountSketch seed 0 (OLS, AR(1) rho=0.5 rows)"
                        % (workload, n, d, m, s),
            "l2": "inputs larger than L2 (A = %.2f GB FP32)" % (n * d * 4 / 1e9),
            "parallelism": "replicas" if world > 1 else "single GPU"}


def c5_record(ihs, hbm):
    """The large sparse LASSO workload (CSR 10,000,000 x 1000, 5 nonzeros a
    row at Zipf(1.1) columns, FP32 values, SJLT s = 8, m = 10000, l1 ball of
    radius ||x*||_1 / 2, mixed TF32, 20 iterations): the solve (CUDA events,
    median of 3 after a warm-up) and, from a one-stream profile of 5 sketches,
    the CSC sketch kernel's bandwidth on its algorithmic bytes (the column
    copy's values and row indices read once, SA written once)."""
    import torch
    w = synth.make("lasso_csr_zipf", seed=0)
    n, d, m, s = w["n"], w["d"], w["m"], w["s"]
    rp, col, val = (torch.from_numpy(w[k]).cuda() for k in ("rowptr", "col", "val"))
    b = torch.from_numpy(w["b"]).cuda()
    kw = dict(kind="l1", param=w["param"], m=m, s=s, seed=0, precision=w["precision"],
              shape=(n, d))
    t0 = time.perf_counter()
    sv = ihs.IHS((rp, col, val), b, **kw)
    torch.cuda.synchronize()
    create_ms = (time.perf_counter() - t0) * 1e3
    iters = w["iters"]
    x0 = torch.zeros(d, dtype=torch.float64, device="cuda")
    sv.solve(x0.clone(), iters=iters)
    times = []
    for _ in range(3):
        x = x0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, rep = sv.solve(x, iters=iters)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    sv.close()
    del sv
    sv = ihs.IHS((rp, col, val), b, serial=True, **kw)
    sv.sketch(0)
    sv.profile(True)
    for t in range(1, 6):
        sv.sketch(t)
    ms, cnt, _ = sv.profile_read()
    sv.close()
    del sv
    sk = ms["sketch"] / max(1, cnt["sketch"])
    nnz = int(val.numel())
    alg = nnz * (val.element_size() + 4) + m * d * 4
    return {"workload": "lasso_csr_zipf n=%d d=%d nnz=%d m=%d s=%d l1 ball tf32" % (n, d, nnz, m, s),
            "iters": iters, "solve_ms_median": round(statistics.median(times), 3),
            "solve_ms_all": [round(t, 3) for t in times], "status": int(rep.status),
            "create_ms": round(create_ms, 1),
            "sketch_kernel": "k_sketch_csc_cta (+ k_sketch_csc_merge)",
            "sketch_ms": round(sk, 4),
            "sketch_algorithmic_bytes": alg,
            "sketch_GB_s": round(alg / (sk * 1e-3) / 1e9, 1),
            "sketch_frac": round(alg / (sk * 1e-3) / 1e9 / hbm, 3)}


def run_reference(args, rank, world):
    """The oracle (plain FP64 CPU IHS, the multi-core build of its C loops on
    every host core) as the reference arm, on the same workload and metric:
    each timed step runs as many oracle iterations as fit in --ref-step-budget
    seconds (the mean iteration times the iteration count is the step's time
    to 1e-10; the iteration count is the oracle's own, from a proxy of the
    workload with the same m / d and design)."""
    if rank != 0:
        return None
    nrows = args.cpu_rows
    w = synth.make(args.workload, n=nrows, seed=0)
    w["n"] = synth.WORKLOADS[args.workload]["n"] if args.n is None else args.n
    w["A64"] = np.ascontiguousarray(w["A"], dtype=np.float64)
    T = oracle_iterations_proxy()
    cores, model = host_cpu()
    vals = []
    spent = 0.0
    desc, used = "", 1
    for it in range(args.warmup + args.steps):
        timed_step = it >= args.warmup
        ms, desc, sp, used, _ = oracle_time_to_tol(
            w, nrows, T, iters=1, threads=cores,
            budget_s=args.ref_step_budget if timed_step else None)
        spent += sp
        if timed_step:
            vals.append(ms)
    v = round(statistics.mean(vals), 1)
    return {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(args.workload, w["n"], w["d"], w["m"], w["s"], world),
        "precision": "fp64 (the oracle)",
        "iters_to_1e-10": {"oracle_proxy": T},
        "cpu_baseline": {"value": v, "unit": "ms", "cores": used, "kind": "oracle",
                         "sample": desc, "cpu_seconds": round(spent, 2), "host_cores": cores,
                         "cpu_model": model},
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_oracle_timing(args):
    """The FP64 oracle timed on this host's cores, config by config: the
    20000 x 50 OLS and 1,000,000 x 200 LASSO solves in full; the
    1,048,576 x 500 OLS, 262,144 x 256 ridge and 10,000,000 x 1000 LASSO ones
    over their first two iterations, extrapolated to the iteration count (an
    iteration's cost does not depend on t).  Each runs on one thread and on
    every host core (the OpenMP build of the oracle's C loops, bit-identical
    results); the l1 QP and the d x d solves are numpy's, on whatever threads
    its BLAS uses.  One JSON line per (workload, threads)."""
    import oracle as O
    cores, model = host_cpu()
    plan = [("ols_dense_fp64", None), ("lasso_csr_fp64", None), ("ols_dense_ar1", 2),
            ("ridge_dense", 2), ("lasso_csr_zipf", 2)]
    if args.only:
        plan = [p for p in plan if p[0] in args.only.split(",")]
    for name, part in plan:
        w = synth.make(name, seed=0)
        if "A" in w:
            A = np.ascontiguousarray(w["A"], dtype=np.float64)
        else:
            A = O.CSR(w["n"], w["d"], w["rowptr"], w["col"], np.asarray(w["val"], dtype=np.float64))
        kind = {"ols": O.OLS, "l1": O.L1_BALL, "ridge": O.RIDGE}[w["kind"]]
        T = w["iters"] or 25
        run = T if part is None else part
        for threads in sorted({1, cores}):
            used = O.use_threads(threads)
            t0 = time.perf_counter()
            O.ihs(A, w["b"], kind, w["param"], w["m"], w["s"], 0, run)
            sec = time.perf_counter() - t0
            print(json.dumps({
                "experiment": "oracle_timing", "workload": name, "n": w["n"], "d": w["d"],
                "m": w["m"], "s": w["s"], "threads": used, "host_cores": cores, "cpu_model": model,
                "iters_run": run, "iters_total": T, "ms_per_iter": round(sec * 1e3 / run, 1),
                "ms_solve": round(sec * 1e3 / run * T, 1),
                "how": "measured whole solve" if part is None else "two iterations, extrapolated"}),
                flush=True)


def run_iters_only(args):
    """Profiling driver: create the solver on the workload and run exactly
    args.ncu_iters iterations (no x_OPT, no timing).  Used under ncu."""
    import torch
    import paper_1910_14166_gb300 as ihs
    w = synth.make(args.workload, n=args.n, seed=0)
    prec = args.precision if args.precision_given else w["precision"]
    b = torch.from_numpy(w["b"]).cuda()
    if "A" in w:
        A, shape = torch.from_numpy(w["A"]).cuda(), None
    else:
        A = tuple(torch.from_numpy(w[k]).cuda() for k in ("rowptr", "col", "val"))
        shape = (w["n"], w["d"])
    kind = args.kind or {"ols": "ols", "l1": "l1", "ridge": "ridge"}[w["kind"]]
    param = w["param"] if args.param is None else args.param
    sv = ihs.IHS(A, b, kind=kind, param=param, m=w["m"], s=w["s"], seed=0, precision=prec,
                 shape=shape, sketch=args.sketch)
    x, rep = sv.solve(iters=args.ncu_iters)
    torch.cuda.synchronize()
    print("iters_only ok: %s n=%d d=%d m=%d s=%d precision=%s kind=%s sketch=%s iters=%d status=%d"
          % (args.workload, w["n"], w["d"], w["m"], w["s"], prec, kind, args.sketch, args.ncu_iters,
             rep.status))


def run_sketch_quality(args):
    """The sketch-quality experiment of App. B on a synthetic stand-in: for
    m in {5d, 10d, 20d, 40d} and s in {1, 4, 8}, the mean and spread over
    `trials` independent sketches of ||A^T S^T S A - A^T A||_F / ||A^T A||_F
    (and the SRHT at the same m on dense data, the paper's comparison),
    and the time to form one sketched Hessian (sort, SA, fix-up, Gram; CUDA
    events).  A^T A, every sketch, every Gram and the error reduction run in
    the library's kernels.  One JSON line per (m, s)."""
    import torch
    import paper_1910_14166_gb300 as ihs
    w = synth.make(args.workload, n=args.n, seed=0)
    prec = args.precision if args.precision_given else "fp64"
    n, d = w["n"], w["d"]
    b = torch.from_numpy(w["b"]).cuda()
    if "A" in w:
        A, shape = torch.from_numpy(w["A"]).cuda(), None
    else:
        A = tuple(torch.from_numpy(w[k]).cuda() for k in ("rowptr", "col", "val"))
        shape = (n, d)
    G = None
    kinds = [("sparse", 1), ("sparse", 4), ("sparse", 8)]
    if shape is None:
        kinds += [("srht", 1), ("gaussian", 1)]
    if args.families:
        kinds = [kv for kv in kinds if kv[0] in args.families.split(",")]
    for sketch, s in kinds:
        for k in (5, 10, 20, 40):
            m = k * d
            if m % s or m > n:
                continue
            # the Gaussian sketch is a dense m x n x d product: keep its FP64
            # form to problems where one sketch is a fraction of a second
            if sketch == "gaussian" and prec == "fp64" and 2.0 * m * n * d > 2e11:
                continue
            try:
                sv = ihs.IHS(A, b, m=m, s=s, seed=args.seed, precision=prec, shape=shape,
                             sketch=sketch)
            except ihs.IHSError as e:
                print(json.dumps({"experiment": "sketch_quality", "workload": args.workload, "m": m,
                                  "s": s, "sketch": sketch, "skipped": str(e)}), flush=True)
                continue
            if G is None:
                G = sv.exact_gram()
                torch.cuda.synchronize()
                # closed form of E err^2 (dense A): (||A||_F^4 + ||A^T A||_F^2
                # - 2 sum_i ||a_i||^4) / (m ||A^T A||_F^2), CountSketch and SJLT
                c_num = None
                if shape is None:
                    row2 = (A.double() ** 2).sum(dim=1)
                    g2 = float((G * G).sum())
                    c_num = (float(row2.sum()) ** 2 + g2 - 2.0 * float((row2 * row2).sum())) / g2
            sv.sketch_error(0, G)  # warm-up
            sv.profile(True)
            errs = [sv.sketch_error(t, G) for t in range(args.trials)]
            ms, cnt, _ = sv.profile_read()
            per = (ms["sort"] + ms["sketch"] + ms["sketch_fix"] + ms["gram"]) / args.trials
            print(json.dumps({
                "experiment": "sketch_quality", "workload": args.workload, "n": n, "d": d,
                "m": m, "m_over_d": k, "s": s, "sketch": sketch, "precision": prec,
                "trials": args.trials,
                "err_mean": statistics.fmean(errs), "err_std": statistics.stdev(errs),
                "sketch_ms": per,
                "err_rms_expected": ((c_num / m) ** 0.5 if c_num is not None and sketch == "sparse"
                                     else None),
                "err_rms": statistics.fmean([e * e for e in errs]) ** 0.5,
                "error": "||A^T S^T S A - A^T A||_F / ||A^T A||_F (App. B)"}), flush=True)
            del sv


def run_adjoint(args):
    """The differentiation form on the 262144 x 256 ridge workload: solve to
    1e-10 (mixed), then the adjoint of L = ||x - x_target||^2 through
    ihs_adjoint: PCG with the sketched factor, dL/db and dL/dA.  CUDA events
    around the call, median of `--steps` runs after one warm-up, with and
    without dL/dA (the difference is the dL/dA pass: read A, write dL/dA).
    One JSON line."""
    import torch
    import paper_1910_14166_gb300 as ihs
    w = synth.make("ridge_dense", n=args.n)
    n, d, m = w["n"], w["d"], w["m"]
    A = torch.from_numpy(w["A"]).cuda()
    b = torch.from_numpy(w["b"]).cuda()
    xt = torch.from_numpy(w["x_target"]).cuda()
    sv = ihs.IHS(A, b, kind="ridge", param=w["param"], m=m, s=1, seed=0, precision="tf32")
    x, _ = sv.solve(iters=40)
    dLdx = 2.0 * (x - xt)
    st = torch.cuda.current_stream()

    def timed(want_A):
        ts, cg = [], 0
        for it in range(1 + args.steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            _, _, rep = sv.adjoint(x, dLdx, want_A=want_A)
            e1.record(st)
            torch.cuda.synchronize()
            cg = rep.iters
            if it >= 1:
                ts.append(e0.elapsed_time(e1))
        return statistics.median(ts), cg

    ms_full, cg = timed(True)
    ms_b, _ = timed(False)
    hbm, hbm_kind = peaks()
    dA_ms = max(ms_full - ms_b, 1e-6)
    dA_bytes = 2 * n * d * 4 + n * 8 * 2  # read A, write dL/dA, b and the residual pass's vectors
    print(json.dumps({
        "experiment": "adjoint", "workload": "ridge_dense n=%d d=%d m=%d lambda=%g tf32" % (
            n, d, m, w["param"]),
        "cg_iters": cg, "adjoint_ms": round(ms_full, 3), "adjoint_no_dLdA_ms": round(ms_b, 3),
        "dLdA_pass_ms": round(dA_ms, 4), "dLdA_GB_s": round(dA_bytes / (dA_ms * 1e-3) / 1e9, 1),
        "dLdA_frac_of_hbm": round(dA_bytes / (dA_ms * 1e-3) / 1e9 / hbm, 3), "peak_kind": hbm_kind,
        "pass_bytes": n * d * 4}), flush=True)


def run_workloads(args):
    """Time every workload of the suite (and the penalised-LASSO form on the
    two sparse ones, lambda = 5; the SRHT and Gaussian comparison sketches and
    the p = 2 ball of radius ||x*|| / 2 on the two dense OLS ones) through
    ihs_solve: CUDA events around the
    call, median of `--steps` runs after one warm-up, plus the library's stage
    times (one serial-mode run: every stage on one stream) and launch count.
    The dense 1,048,576 x 500 OLS line is the main benchmark's step.  One JSON
    line per case."""
    import torch
    import paper_1910_14166_gb300 as ihs
    cases = [("ols_dense_fp64", None, None, "sparse"), ("lasso_csr_fp64", None, None, "sparse"),
             ("ols_dense_ar1", None, None, "sparse"), ("ridge_dense", None, None, "sparse"),
             ("lasso_csr_zipf", None, None, "sparse"), ("lasso_csr_fp64", "l1pen", 5.0, "sparse"),
             ("lasso_csr_zipf", "l1pen", 5.0, "sparse"), ("ols_dense_fp64", None, None, "srht"),
             ("ols_dense_ar1", None, None, "srht"), ("ols_dense_fp64", None, None, "gaussian"),
             ("ols_dense_ar1", None, None, "gaussian"), ("ols_dense_fp64", "l2", "half", "sparse"),
             ("ols_dense_ar1", "l2", "half", "sparse")]
    for name, kind_o, param_o, sketch in cases:
        if args.only and name not in args.only.split(","):
            continue
        w = synth.make(name, seed=0)
        b = torch.from_numpy(w["b"]).cuda()
        if "A" in w:
            A, shape = torch.from_numpy(w["A"]).cuda(), None
        else:
            A = tuple(torch.from_numpy(w[k]).cuda() for k in ("rowptr", "col", "val"))
            shape = (w["n"], w["d"])
        kind = kind_o or {"ols": "ols", "l1": "l1", "ridge": "ridge"}[w["kind"]]
        param = w["param"] if param_o is None else param_o
        if param_o == "half":  # p = 2 ball of radius ||x*|| / 2 (the constraint active)
            param = 0.5 * float(np.linalg.norm(w["x_star"]))
        iters = w["iters"] or 25
        times, times_ng, used_graph = [], [], False
        for serial, graph in ((False, True), (False, False), (True, False)):
            if not serial and not graph and not used_graph:
                continue  # the context replays no graph anyway
            sv = ihs.IHS(A, b, kind=kind, param=param, m=w["m"], s=w["s"], seed=0,
                         precision=w["precision"], shape=shape, serial=serial, sketch=sketch,
                         graph=graph)
            x0 = torch.zeros(w["d"], dtype=torch.float64, device="cuda")
            sv.solve(x0.clone(), iters=iters)  # warm-up (and graph capture)
            if serial:
                sv.profile(True)
                sv.solve(x0.clone(), iters=iters)
                ms, cnt, launches = sv.profile_read()
                stages = {k: round(v / iters, 4) for k, v in ms.items()}
            else:
                out = times if graph else times_ng
                for _ in range(max(1, args.steps)):
                    x = x0.clone()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record()
                    _, rep = sv.solve(x, iters=iters)
                    e1.record()
                    torch.cuda.synchronize()
                    out.append(e0.elapsed_time(e1))
                    if graph:
                        status, fista, used_graph = rep.status, rep.qp_fista_iters, bool(rep.graph)
            del sv
        print(json.dumps({
            "experiment": "workloads", "workload": name, "kind": kind, "param": param, "sketch": sketch,
            "n": w["n"], "d": w["d"], "m": w["m"], "s": w["s"], "precision": w["precision"],
            "iters": iters, "solve_ms_median": statistics.median(times), "solve_ms_all": times,
            "graph": used_graph,
            "solve_ms_median_no_graph": statistics.median(times_ng) if times_ng else None,
            "status": status, "qp_fista_iters": fista, "stage_ms_per_iter_serial": stages,
            "launches_per_solve": launches}), flush=True)
        del A, b


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ols_dense_ar1")
    ap.add_argument("--precision", default="tf32", choices=["tf32", "bf16", "fp64"])
    ap.add_argument("--ncu-iters", type=int, default=0,
                    help="profiling driver: run this many iterations and exit")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--cpu-rows", type=int, default=None,
                    help="rows of the workload the CPU oracle is timed on (default: all)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-two-pass", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the Gaussian-sketch and sparse-LASSO records")
    ap.add_argument("--ref-step-budget", type=float, default=15.0,
                    help="reference arm: seconds of oracle iterations per timed step")
    ap.add_argument("--cpu-budget", type=float, default=40.0,
                    help="seconds of oracle iterations the CPU baseline may run (whole solve "
                         "when it fits)")
    ap.add_argument("--only", default=None, help="workloads experiment: comma-separated names")
    ap.add_argument("--experiment", default=None, choices=["sketch-quality", "workloads", "adjoint", "c5", "oracle-timing"],
                    help="run an experiment instead of the benchmark (one JSON line per point)")
    ap.add_argument("--trials", type=int, default=10)
    ap.add_argument("--families", default=None,
                    help="sketch-quality: comma list of sparse, srht, gaussian (default all)")
    ap.add_argument("--sketch", default="sparse", choices=["sparse", "srht", "gaussian"],
                    help="profiling driver: sketch family")
    ap.add_argument("--kind", default=None, choices=["ols", "l1", "l1pen", "l2", "ridge"],
                    help="profiling driver: constraint (default: the workload's)")
    ap.add_argument("--param", type=float, default=None,
                    help="profiling driver: constraint parameter (default: the workload's)")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    args.precision_given = any(a == "--precision" or a.startswith("--precision=") for a in sys.argv[1:])
    if args.ncu_iters:
        run_iters_only(args)
        return
    if args.experiment == "sketch-quality":
        run_sketch_quality(args)
        return
    if args.experiment == "workloads":
        run_workloads(args)
        return
    if args.experiment == "adjoint":
        run_adjoint(args)
        return
    if args.experiment == "oracle-timing":
        run_oracle_timing(args)
        return
    if args.experiment == "c5":  # the large sparse LASSO record of the main line, alone
        import paper_1910_14166_gb300 as ihs
        print(json.dumps(dict(experiment="c5", **c5_record(ihs, peaks()[0]))), flush=True)
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1 and args.impl == "ours":
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    res = run_reference(args, rank, world) if args.impl == "reference" else run_ours(args, rank, world)
    if rank == 0 and res is not None:
        print(json.dumps(res), flush=True)
    if world > 1 and args.impl == "ours":
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
