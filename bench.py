"""Benchmark: batched OMP signals/s on one GB300 (or N replicas under torchrun).

A step is one whole solve (every OMP iteration: correlate, select, append, update, compact,
finalize) of the batch through the C ABI, graph-replayed, with the dictionary prepared and the
signals resident in HBM before the timed region. Workload: the 1024 x 8192 Gaussian dictionary,
B = 4096 planted 32-sparse signals with noise sigma = 1e-3, S = 32 fixed iterations. The chosen
form (BF16 tensor-core correlation with FP32 top-8 rescoring) is timed next to the plain FP32
path on the same GPU; the L2 is flushed (a 512 MiB write) between timed steps.

Roofline: the dominant kernel's per-launch duration comes from CUDA events recorded around
every correlation / update launch inside an instrumented replay of the same graph
(omp_profile_*); algorithmic FLOPs / bytes per launch are derived from the live counts.

``--impl reference`` times the FP64 CPU oracle (timed mode) on the host cores instead, each step
a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from workloads import gen  # noqa: E402

WORKLOAD = "gaussian_1024x8192_s32_b4096"
METRIC = "OMP signals/s, chosen form vs plain FP32 on same GB300 at matched support; % roofline"
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu capture of the same
# kernel source at full live count (profiles/<kernel>_<workload>.md gives the command); ncu
# flushes the caches before the capture, so this is the cold-cache traffic of one launch. An
# entry is removed whenever its kernel changes.
L2_RESIDENT_BYTES = 64 << 20   # an FP32 dictionary up to half the 129 MB L2 stays resident
MEASURED_TRAFFIC = {
    ("gaussian_1024x8192_s32_b4096", "bf16", "correlate"): 25316864.0,
    ("gaussian_1024x8192_s32_b4096", "bf16", "update"): 61508864.0,
}
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
# FP32 non-tensor peak: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz (nominal unit counts)
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_batch(w, A, rank: int):
    """Rank r's shard of a weak-scaling run: the workload's batch drawn with seed r, so rank 0
    solves exactly the single-GPU batch and every rank a distinct one of the same shape (signals
    are independent, so ranks share no data and need no collective on the solve path)."""
    Y, *_ = gen.signals(w, A, seed=rank)
    return Y


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The slowest rank's value (the whole job ends with it); the identity on one rank."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def oracle_cores():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads", 0) for i in threadpool_info() if i.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


_ORACLE_CACHE = {}


def time_oracle(w, A, Y, seconds_target=15.0, max_signals=None):
    """FP64 timed-mode oracle on a bounded sample: grows the sample until ~seconds_target."""
    from oracle import omp as oracle_omp
    n = 16
    total_t, total_n = 0.0, 0
    while True:
        rows = slice(0, min(n, Y.shape[0]))
        t0 = time.perf_counter()
        ref = oracle_omp.omp_batch(A, Y[rows], w.S, w.eps, True)
        dt = time.perf_counter() - t0
        total_t, total_n = dt, rows.stop
        _ORACLE_CACHE[(w.name, rows.stop)] = ref
        if total_t >= seconds_target / 4 or rows.stop >= Y.shape[0] or \
                (max_signals and rows.stop >= max_signals):
            break
        n *= 2
    return total_n / total_t, total_n, total_t


def accuracy_report(w, A, Y, n, res):
    """Errors of a solve's results against the FP64 oracle on the first n signals of the batch:
    per-signal coefficient error ||x - x_ref|| / ||x_ref|| (max and median), residual-norm error
    (max relative, and max over its tolerance 1e-4 ||r|| + 1e-6 ||y||), supports that differ at a
    top-two margin above 1e-3 (must be 0), near-tie divergences, with the parity rules of the
    tests (a diverged signal is measured against the least squares on its own support)."""
    from oracle import compare
    from oracle import omp as oracle_omp
    key = (w.name, n)
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = oracle_omp.omp_batch(A, Y[:n], w.S, w.eps, True)
    ref = _ORACLE_CACHE[key]
    st = compare.compare(A, Y[:n], ref, res["sup"][:n], res["X"][:n], res["n_iter"][:n],
                         res["resid"][:n], eps=w.eps, strict=False)
    rep = compare.error_report(st)
    rep["reference"] = f"FP64 oracle, first {n} signals of the batch"
    return rep


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2407_06434_gb300 import omp

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = gen.get_config(args.config)
    A = gen.dictionary(w)
    Y = rank_batch(w, A, rank)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t()
    Yd = torch.from_numpy(Y).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def bench_form(prec, gather24=False):
        solver = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision=prec,
                               gather24=gather24)
        h = solver.h
        X = torch.empty((w.B, w.S), dtype=torch.float32, device=dev)
        sup = torch.empty((w.B, w.S), dtype=torch.int32, device=dev)
        omp.omp_prepare_dictionary(h, Ad)
        tuned = omp.omp_autotune(h, Ad, Yd, w.S, w.eps, repeats=4)
        shapes = omp.omp_tuning(h)
        for _ in range(args.warmup):
            omp.omp_solve_batch(h, Ad, Yd, w.S, w.eps, X, sup)
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            starts[i].record(stream)
            omp.omp_solve_batch(h, Ad, Yd, w.S, w.eps, X, sup)
            ends[i].record(stream)
        torch.cuda.synchronize()
        barrier()
        ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        total = max_over_ranks(sum(ms), world, dev)
        # instrumented replay: per-launch durations of correlation and update kernels
        omp.omp_profile_enable(h, True)
        corr = np.zeros(w.S)
        upd = np.zeros(w.S)
        live = None
        for i in range(max(1, min(args.steps, 5))):
            flush.zero_()
            omp.omp_solve_batch(h, Ad, Yd, w.S, w.eps, X, sup)
            c, u, lv = omp.omp_profile_read(h, w.S)
            corr += c
            upd += u
            live = lv
            n_prof = i + 1
        omp.omp_profile_enable(h, False)
        corr /= n_prof
        upd /= n_prof
        # end to end through the host entry point (pinned buffers, copies inside)
        Yh = torch.from_numpy(Y).pin_memory()
        Xh = torch.empty((w.B, w.S), dtype=torch.float32).pin_memory()
        Sh = torch.empty((w.B, w.S), dtype=torch.int32).pin_memory()
        omp.omp_solve_batch_host(h, Ad, Yh, w.S, w.eps, Xh, Sh)
        e2e_t = []
        for _ in range(max(3, min(args.steps, 10))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            omp.omp_solve_batch_host(h, Ad, Yh, w.S, w.eps, Xh, Sh)
            e2e_t.append(time.perf_counter() - t0)
        # one more solve, untimed, with the per-signal diagnostics the error report uses
        Xd, Sd, nd, rd, _ = solver.solve(Ad, Yd, w.S, w.eps, diagnostics=True)
        torch.cuda.synchronize()
        res = dict(total_ms=total, ms=ms, corr=corr, upd=upd, live=live, update_warps=tuned, shapes=shapes,
                   e2e_s=float(np.sum(e2e_t)), e2e_steps=len(e2e_t),
                   sup=Sd.cpu().numpy(), X=Xd.cpu().numpy(), n_iter=nd.cpu().numpy(),
                   resid=rd.cpu().numpy())
        solver.close()
        return res

    with Clocks(local) as clk:
        chosen = bench_form(args.precision, args.gather24)
    plain = bench_form("fp32") if args.precision != "fp32" and not args.skip_plain else None
    clocks = clk.summary()
    # L2-to-SM streaming read bandwidth (the library's probe kernel, 64 MiB buffer), measured
    # after the timed work: the update kernel's roofline when the FP32 dictionary fits in L2
    l2_gbs = omp.read_bandwidth_gbs(64, 50)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    peaks, peak_src = load_peaks()
    B_all = w.B * world
    value = B_all * args.steps / (chosen["total_ms"] / 1e3)
    # roofline: dominant kernel of the chosen form
    live = chosen["live"].astype(np.float64)
    corr_ms, upd_ms = chosen["corr"], chosen["upd"]
    flops_corr = 2.0 * w.M * w.N * live                    # per launch
    k = np.arange(w.S)
    qbytes = 4 if args.precision == "fp32" else 0
    topk = 1 if args.precision == "fp32" else 8
    # update: gather of k+1 atom rows (4 bytes an element, 3 with the 24-bit copy) + topk FP32
    # rescoring rows (quantised paths) + residual read and write, per live signal
    gb = 3.0 if args.gather24 else 4.0
    upd_bytes = live * w.M * (gb * (k + 1) + 4.0 * ((topk if topk > 1 else 0) + 2))
    if corr_ms.sum() >= upd_ms.sum():
        dur = corr_ms.mean() / 1e3
        achieved = float(flops_corr.mean() / dur / 1e12)
        if args.precision == "fp32":
            peak, unit, bound, src = FP32_SIMT_PEAK_TFLOPS, "TFLOP/s", "alu", "nominal"
        else:
            # each correlation launch is timed on its own (tens of microseconds inside a solve of
            # a few milliseconds), so the burst peak applies; FP8 takes 2x (the nominal ratio)
            key = "bf16_tflops"
            peak = peaks.get(key, PEAKS_FALLBACK[key]) * (2.0 if args.precision == "fp8" else 1.0)
            unit, bound, src = "TFLOP/s", "tensor", peak_src + (" burst" + (" x2 (fp8)" if
                                                                           args.precision == "fp8" else ""))
        kern = "correlate"
        alg = float(flops_corr.mean())
    else:
        dur = upd_ms.mean() / 1e3
        achieved = float(upd_bytes.mean() / dur / 1e9)
        peak, unit, bound, src = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"]), "GB/s", "hbm", \
            peak_src
        kern = "update"
        alg = float(upd_bytes.mean())
    traffic = MEASURED_TRAFFIC.get((w.name, args.precision, kern))
    mp = (w.M + 63) // 64 * 64
    a32_bytes = w.N * mp * 4
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic, "kernel": kern,
                "peak_source": src, "algorithmic_per_launch": alg,
                "launch_ms": float(dur * 1e3),
                "corr_ms_per_step": float(corr_ms.sum()), "update_ms_per_step": float(upd_ms.sum())}
    if kern == "update":
        # the gathered atom rows come from L2 wherever the FP32 dictionary (or most of it) fits
        # there, so the HBM fraction above overstates the kernel; the L2 read peak bounds it
        roofline["l2_read_peak_gbs"] = l2_gbs
        roofline["l2_frac"] = achieved / l2_gbs
        roofline["a32_l2_resident"] = bool(a32_bytes <= L2_RESIDENT_BYTES)
    e2e_value = B_all * chosen["e2e_steps"] / chosen["e2e_s"]
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "signals/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": chosen["total_ms"] / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32": "f32", "bf16": "bf16", "fp8": "fp8_e4m3"}[args.precision],
        "data": "synthetic (seeded Gaussian dictionary and planted sparse signals)",
        "config": {"workload": w.name, "M": w.M, "N": w.N, "B": w.B, "S": w.S,
                   "precision": args.precision, "rescore_topk": topk,
                   "update_warps_per_signal": chosen["update_warps"],
                   "update_persistent": bool(chosen["shapes"][1]),
                   "correlation_stages": chosen["shapes"][2] or None,
                   "correlation_ctas": chosen["shapes"][3] or None,
                   "correlation_cluster": chosen["shapes"][4] or None,
                   "update_gather": "24-bit copy of A (3 bytes an element)" if args.gather24
                   else "FP32 rows",
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": f"replicas{world}" if world > 1 else "single"},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": "signals/s",
                "h2d_bytes_per_step": int(w.B * w.M * 4),
                "d2h_bytes_per_step": int(w.B * w.S * 8)},
        "gpu_launches": int(args.steps * (3 * w.S + 3)),
        "roofline": roofline,
    }
    if plain is not None:
        pv = B_all * args.steps / (plain["total_ms"] / 1e3)
        same = float(np.mean(np.all(plain["sup"] == chosen["sup"], axis=1)))
        line["plain_fp32"] = {"value": pv, "ms_per_step": plain["total_ms"] / args.steps,
                              "corr_ms_per_step": float(plain["corr"].sum()),
                              "update_ms_per_step": float(plain["upd"].sum()),
                              "support_match_rate": same}
        line["speedup_vs_plain_fp32"] = value / pv
    if not args.no_cpu_baseline:
        v, n, t = time_oracle(w, A, Y, seconds_target=args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": "signals/s", "cores": oracle_cores(),
                                "kind": "oracle",
                                "sample": f"first {n} signals of the batch, FP64 timed-mode "
                                          f"oracle, {t:.1f} s"}
        # each result's error against the FP64 oracle, on the same signals (or more)
        n_err = max(n, min(args.error_signals, w.B))
        line["accuracy"] = accuracy_report(w, A, Y, n_err, chosen)
        if plain is not None:
            line["plain_fp32"]["accuracy"] = accuracy_report(w, A, Y, n_err, plain)
    elif args.error_signals > 0:
        line["accuracy"] = accuracy_report(w, A, Y, min(args.error_signals, w.B), chosen)
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def run_gram(args):
    """Gram-space form (omp_solve_batch_gram: one FP32 GEMM for c = A^T y, then per-step updates
    of c through the Gram matrix) on the given workload, next to the dense BF16 form on the same
    batch. Both are timed per solve with CUDA events, L2 flushed between solves; e2e times the
    Gram solve through the Python binding with the batch copied from pinned host memory and the
    coefficients and supports copied back inside the timed region."""
    import torch
    from paper_2407_06434_gb300 import omp

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = gen.get_config(args.config)
    A = gen.dictionary(w)
    Y, *_ = gen.signals(w, A)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t()
    Yd = torch.from_numpy(Y).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    solver = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="bf16")

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = fn()
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return ms, out

    with Clocks(local) as clk:
        g_ms, (Xg, Sg, ng, _, _) = timed(lambda: solver.solve_gram(Ad, Yd, w.S, w.eps, diagnostics=True))
        d_ms, (Xd, Sd) = timed(lambda: solver.solve(Ad, Yd, w.S, w.eps))
    clocks = clk.summary()
    l2_gbs = omp.read_bandwidth_gbs(64, 50)
    Yh = torch.from_numpy(Y).pin_memory()
    Xh = torch.empty((w.B, w.S), dtype=torch.float32).pin_memory()
    Sh = torch.empty((w.B, w.S), dtype=torch.int32).pin_memory()
    e2e = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Yg = Yh.to(dev, non_blocking=True)
        X, S_ = solver.solve_gram(Ad, Yg, w.S, w.eps)
        Xh.copy_(X, non_blocking=True)
        Sh.copy_(S_, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    solver.close()
    if rank != 0:
        return
    n_it = ng.cpu().numpy().astype(np.float64)
    gram_bytes = float(np.sum(n_it * (n_it + 1) / 2) * w.N * 4)   # Gram rows read by the c updates
    total = float(np.sum(g_ms))
    value = w.B * args.steps / (total / 1e3)
    achieved = gram_bytes / (np.mean(g_ms) / 1e3) / 1e9
    peaks, src = load_peaks()
    hbm = peaks.get("hbm_gbs", PEAKS_FALLBACK["hbm_gbs"])
    agree = float(np.mean(np.all(Sg.cpu().numpy() == Sd.cpu().numpy(), axis=1)))
    line = {
        "metric": METRIC, "value": value, "unit": "signals/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded Gaussian dictionary and planted sparse signals)",
        "config": {"workload": w.name, "form": "Gram-space (FP32 first correlation, c updated through G)",
                   "M": w.M, "N": w.N, "B": w.B, "S": w.S, "eps": w.eps,
                   "l2": "flushed between timed steps (512 MiB write)"},
        "clocks": clocks,
        "e2e": {"value": w.B * len(e2e) / float(np.sum(e2e)), "unit": "signals/s",
                "h2d_bytes_per_step": int(Y.nbytes), "d2h_bytes_per_step": int(w.B * w.S * 8)},
        "gpu_launches": 5 * args.steps,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "kernel": "gram_solve (whole solve)",
                     "peak_source": src, "algorithmic_per_launch": gram_bytes,
                     "l2_read_peak_gbs": l2_gbs, "l2_frac": achieved / l2_gbs},
        "dense_bf16": {"value": w.B * args.steps / (float(np.sum(d_ms)) / 1e3),
                       "ms_per_step": float(np.mean(d_ms)), "support_agreement": agree},
    }
    print(json.dumps(line))


def run_learned(args):
    """Learned-proposal form on the 1024 x 8192, S = 48, B = 16384 workload: train the proposal
    network on generated signals labelled by plain OMP, then time the learned solve next to the
    dense BF16 solve and the plain FP32 solve on the same batch, and report fallback and
    support-recovery rates."""
    import torch
    from paper_2407_06434_gb300 import omp, proposal as prop

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = gen.get_config(args.config if args.config != WORKLOAD else "gaussian_1024x8192_s48_b16384")
    hidden = args.hidden
    A = gen.dictionary(w)
    Y, sp, planted, _ = gen.signals(w, A)
    Ad = torch.from_numpy(np.ascontiguousarray(A.T)).to(dev).t()
    Yd = torch.from_numpy(Y).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    dense = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="bf16")
    p = omp.Proposal(dense.h, hidden=hidden, topk=256, max_batch=w.B, train_batch=4096,
                     pos_weight=float(w.N - w.S) / w.S, lr=args.train_lr)
    W1, b1, W2, b2, beta = prop.init_weights(w.N, hidden, w.S, seed=0, M=w.M)
    p.set_weights(*[torch.from_numpy(v).to(dev) for v in (W1, b1, W2, b2, beta)])
    rep = prop.train(dense.h, p, Ad, w, n_signals=args.train_signals, epochs=args.train_epochs,
                     batch=4096, chunk=w.B)
    X = torch.empty((w.B, w.S), dtype=torch.float32, device=dev)
    sup = torch.empty((w.B, w.S), dtype=torch.int32, device=dev)
    n_iter = torch.empty(w.B, dtype=torch.int32, device=dev)
    resid = torch.empty(w.B, dtype=torch.float32, device=dev)
    fb = torch.empty(w.B, dtype=torch.int32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ms = []
        for _ in range(args.steps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
        return float(np.sum(ms))

    with Clocks(local) as clk:
        t_learned = timed(lambda: omp.omp_solve_batch_learned(dense.h, p, Ad, Yd, w.S, w.eps, X, sup,
                                                              n_iter, resid, fb))
        sup_l, fb_l = sup.cpu().numpy(), fb.cpu().numpy()
        t_dense = timed(lambda: omp.omp_solve_batch(dense.h, Ad, Yd, w.S, w.eps, X, sup))
        sup_d = sup.cpu().numpy()
        plain = omp.OmpSolver(w.M, w.N, max_batch=w.B, max_iters=w.S, precision="fp32")
        t_plain = timed(lambda: omp.omp_solve_batch(plain.h, Ad, Yd, w.S, w.eps, X, sup))
        sup_p = sup.cpu().numpy()
    clocks = clk.summary()
    # end to end: the batch from pinned host memory, the learned solve, X and supports back
    Yh = torch.from_numpy(Y).pin_memory()
    Xh = torch.empty((w.B, w.S), dtype=torch.float32).pin_memory()
    Sh = torch.empty((w.B, w.S), dtype=torch.int32).pin_memory()
    e2e = []
    for _ in range(max(3, min(args.steps, 10))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Yg = Yh.to(dev, non_blocking=True)
        omp.omp_solve_batch_learned(dense.h, p, Ad, Yg, w.S, w.eps, X, sup, n_iter, resid, fb)
        Xh.copy_(X, non_blocking=True)
        Sh.copy_(sup, non_blocking=True)
        torch.cuda.synchronize()
        e2e.append(time.perf_counter() - t0)
    rec = lambda S_: float(np.mean([set(S_[b][S_[b] >= 0]) == set(planted[b]) for b in range(w.B)]))
    # what the network gains over the same method without it (candidates = top-K of |A^T y|):
    # recall of plain OMP's picks among the candidates, the fallback steps, and the time of each
    # part (network inference alone; the candidate-restricted solve with its dense fallback)
    K = p.desc.topk
    cm = torch.empty((w.B, K), dtype=torch.int32, device=dev)
    cb = torch.empty((w.B, K), dtype=torch.int32, device=dev)
    t_infer = timed(lambda: p.infer(Ad, Yd, cm))
    t_base_cand = timed(lambda: p.baseline_candidates(Ad, Yd, cb))
    tau_d = torch.from_numpy(np.asarray(rep.tau, dtype=np.float32)).to(dev)
    fb_b = torch.empty(w.B, dtype=torch.int32, device=dev)

    def solve_cands(c, fbo):
        omp.omp_solve_batch_candidates(dense.h, Ad, Yd, w.S, w.eps, c, tau_d, X, sup, n_iter, resid, fbo)

    t_cand_m = timed(lambda: solve_cands(cm, fb))
    fbm = fb.cpu().numpy()
    t_cand_b = timed(lambda: solve_cands(cb, fb_b))
    fbb = fb_b.cpu().numpy()
    cm_h, cb_h = cm.cpu().numpy(), cb.cpu().numpy()
    recall = lambda C: float(np.mean([np.isin(sup_p[b][sup_p[b] >= 0], C[b]).mean() for b in range(w.B)]))
    # the step at which plain OMP first needs an atom that is not a candidate (S if never)
    def first_miss(C):
        out = np.full(w.B, w.S)
        for b in range(w.B):
            miss = np.flatnonzero(~np.isin(sup_p[b], C[b]) & (sup_p[b] >= 0))
            if miss.size:
                out[b] = miss[0]
        return out
    edges = list(range(0, w.S + 8, 8))
    hist = lambda f: np.histogram(np.where(f >= 0, f, w.S), bins=edges)[0].tolist()
    gain = {"topk": K, "tau_quantile": 1e-3,
            "recall_of_plain_picks": {"learned": recall(cm_h), "no_network": recall(cb_h)},
            "first_missing_pick_step_mean": {"learned": float(first_miss(cm_h).mean()),
                                             "no_network": float(first_miss(cb_h).mean())},
            "fallback_rate": {"learned": float(np.mean(fbm >= 0)), "no_network": float(np.mean(fbb >= 0))},
            "mean_fallback_step": {"learned": float(np.mean(np.where(fbm >= 0, fbm, w.S))),
                                   "no_network": float(np.mean(np.where(fbb >= 0, fbb, w.S)))},
            "fallback_step_histogram": {"bins": edges, "learned": hist(fbm), "no_network": hist(fbb)},
            "ms_per_solve": {"network_inference": t_infer / args.steps,
                             "no_network_candidates": t_base_cand / args.steps,
                             "restricted_and_fallback_learned": t_cand_m / args.steps,
                             "restricted_and_fallback_no_network": t_cand_b / args.steps,
                             "dense_bf16": t_dense / args.steps}}
    value = w.B * args.steps / (t_learned / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "signals/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_learned / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
        "data": "synthetic (seeded Gaussian dictionary, planted sparse signals)",
        "config": {"workload": w.name, "form": "learned proposal (top-256) + BF16 fallback",
                   "M": w.M, "N": w.N, "B": w.B, "S": w.S, "l2": "flushed between timed steps",
                   "train_signals": args.train_signals, "train_epochs": args.train_epochs,
                   "hidden": hidden, "train_lr": args.train_lr,
                   "supports": (f"blocks of {w.group} consecutive atoms" if w.group > 1
                                else "uniform"), "coefficients": w.coef_kind},
        "clocks": clocks,
        "e2e": {"value": w.B * len(e2e) / float(np.sum(e2e)), "unit": "signals/s",
                "h2d_bytes_per_step": int(Y.nbytes), "d2h_bytes_per_step": int(w.B * w.S * 8)},
        "learned": {"fallback_rate": float(np.mean(fb_l >= 0)),
                    "mean_fallback_step": float(np.mean(fb_l[fb_l >= 0])) if np.any(fb_l >= 0) else None,
                    "planted_recovery": rec(sup_l), "support_equal_to_plain": float(np.mean(np.all(sup_l == sup_p, axis=1))),
                    "train_seconds_data": rep.seconds_data, "train_seconds": rep.seconds_train,
                    "train_losses": rep.losses},
        "dense_bf16": {"value": w.B * args.steps / (t_dense / 1e3), "planted_recovery": rec(sup_d)},
        "network_gain": gain,
        "plain_fp32": {"value": w.B * args.steps / (t_plain / 1e3), "planted_recovery": rec(sup_p)},
    }
    print(json.dumps(line))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import omp as oracle_omp
    w = gen.get_config(args.config)
    A = gen.dictionary(w)
    n = args.reference_signals
    Y, *_ = gen.signals(w, A, rows=slice(0, n))
    for _ in range(args.warmup):
        oracle_omp.omp_batch(A, Y, w.S, w.eps, True)
    t = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_omp.omp_batch(A, Y, w.S, w.eps, True)
        t.append(time.perf_counter() - t0)
    value = n * args.steps / sum(t)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "signals/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * sum(t) / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "M": w.M, "N": w.N, "B": w.B, "S": w.S,
                   "sample_signals_per_step": n},
        "cpu_baseline": {"value": value, "unit": "signals/s", "cores": oracle_cores(),
                         "kind": "oracle",
                         "sample": f"first {n} signals of the batch per step, FP64 timed-mode "
                                   "oracle"},
        "e2e": {"value": value, "unit": "signals/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--gather24", action="store_true",
                    help="the update gathers atom rows from the 24-bit copy of A")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--error-signals", type=int, default=0,
                    help="signals checked against the FP64 oracle for the accuracy report "
                         "(default: the CPU baseline's timed sample)")
    ap.add_argument("--reference-signals", type=int, default=64)
    ap.add_argument("--form", default="dense", choices=["dense", "learned", "gram"])
    ap.add_argument("--train-signals", type=int, default=1 << 20)
    ap.add_argument("--train-epochs", type=int, default=3)
    ap.add_argument("--train-lr", type=float, default=1e-3)
    ap.add_argument("--hidden", type=int, default=1024)
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.form == "learned":
        run_learned(args)
    elif args.form == "gram":
        run_gram(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
