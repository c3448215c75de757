#!/usr/bin/env python
"""Benchmark: AR(p) Toeplitz-LSQR solves/s, FP64 and mixed precision, on one GB300 per rank.

Workload (default): one stationary AR(100) series, n = 2^22, roots of modulus U[1.05, 2], Student-t(5)
innovations scaled to unit variance, FP64 throughout, solved to a normal-equation ratio of 1e-10. A step is
one complete solve (Gram pass, Cholesky preconditioner, LSQR passes, float64 check pass) of that series with
the series already resident in HBM. The same series is also solved in mixed precision, and end to end from
pinned host memory through the C ABI (toeplitz_ols_solve).

Under torchrun every rank solves its own replica (weak scaling, no collective on the data path); value is the
whole-job solves/s with the max time over ranks.

--impl reference times the CPU oracle (float64 Householder QR, NumPy/LAPACK on the host cores) on a bounded
sample of the same workload and prints the same JSON line with "impl": "reference".
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "AR(p) Toeplitz-LSQR solves/s & matvec HBM GB/s, mixed vs FP64; p99 latency"
WORKLOADS = {
    "ar100_n4M": dict(n=1 << 22, p=100, root_lo=1.05, root_hi=2.0, noise="t5", tol=1e-10, config_id=2,
                      desc="AR(100), n=2^22, roots |r| in U[1.05,2], Student-t(5) innovations, FP64, ne-ratio 1e-10"),
    "ar100_n64M": dict(n=1 << 26, p=100, root_lo=1.05, root_hi=2.0, noise="normal", tol=1e-10, config_id=3,
                       desc="AR(100), n=2^26, roots |r| in U[1.05,2], N(0,1) innovations (kernel profiling size)"),
    "ar10_n10k": dict(n=10_000, p=10, root_lo=1.2, root_hi=3.0, noise="normal", tol=1e-12, config_id=1,
                      desc="AR(10), n=10,000, roots |r| in U[1.2,3], N(0,1) innovations, FP64, ne-ratio 1e-12"),
}
L2_FLUSH_BYTES = 512 << 20
BATCH_TOL = 1e-10   # normal-equation ratio for the batched and served fits (as for the AR(100) fit)
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12   # 152 SMs x 2 DFMA (4 flop)/clk/SM x 2.07 GHz max clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="ar100_n4M")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time only the fused product pass (toeplitz_ols_gk_pass), float64 then float32")
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--only", default="", help="kernel-only: comma list of direct_fp64,direct_fp32,fft_fp64,fft_fp32")
    ap.add_argument("--p", type=int, default=0, help="kernel-only: override the order p")
    ap.add_argument("--batch-series", type=int, default=1024,
                    help="series in the batched run (n log-uniform in [1e4, 1e6], p uniform in [5, 200]); 0 = skip")
    ap.add_argument("--lsar-only", action="store_true",
                    help="time only Algorithm LSAR on the bench series (--lsar-lags, --lsar-c)")
    ap.add_argument("--batch-only", action="store_true",
                    help="solve the batch of --batch-series series once in float64 and print its timing (profiling)")
    ap.add_argument("--pacf-lags", type=int, default=120,
                    help="order sweep: PACF lags fitted on the bench series (0 = skip)")
    ap.add_argument("--lsar-lags", type=int, default=120,
                    help="Algorithm LSAR on the bench series: lags 1 .. p_bar (0 = skip)")
    ap.add_argument("--lsar-c", type=int, default=2000, help="Algorithm LSAR: rows sampled per lag")
    ap.add_argument("--rh-sketch", type=int, default=16, help="Repeated Halving: rows of the Gaussian sketch")
    ap.add_argument("--rh-only", action="store_true",
                    help="time only the Repeated Halving variant of LSAR on the bench series")
    ap.add_argument("--srht-only", action="store_true",
                    help="time only Algorithm SRHT for the order-p fit of the bench series (c = --lsar-c rows)")
    ap.add_argument("--serve-requests", type=int, default=400,
                    help="requests in the serving run (n log-uniform in [1e3, 1e7], p log-uniform in [1, 300]); 0 = skip")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "20", "-i", str(self.gpu_index)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower().startswith("active")})
        return {"sm_mhz": statistics.median([r[0] for r in rows]) if rows else None,
                "sm_max_mhz": max(r[1] for r in rows) if rows else None,
                "reasons": reasons, "samples": len(rows)}


def dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Ranks:
    """The ranks of a replica run: a barrier and the max over ranks of a host number, nothing on the data path.

    NCCL when the ranks own GPUs, gloo otherwise (the multi-process CPU tests). With one rank every call is a no-op.
    """

    def __init__(self, world, rank, device=None):
        self.world, self.rank, self.device = world, rank, device
        self.on_gpu = device is not None and device.type == "cuda"
        if world > 1:
            import torch.distributed as tdist
            if self.on_gpu:
                tdist.init_process_group("nccl", device_id=device)
            else:
                tdist.init_process_group("gloo")

    def barrier(self):
        if self.world > 1:
            import torch.distributed as tdist
            tdist.barrier()

    def max(self, x):
        if self.world == 1:
            return x
        import torch
        import torch.distributed as tdist
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device if self.on_gpu else "cpu")
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.world > 1:
            import torch.distributed as tdist
            tdist.destroy_process_group()


def whole_job_rate(world, units_per_rank, max_seconds):
    """Units all ranks processed divided by the slowest rank's time (every rank does the same work)."""
    return world * units_per_rank / max_seconds


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        if info:
            return max(i.get("num_threads", 0) for i in info)
    except Exception:
        pass
    return os.cpu_count()


def _gen_one(args):
    from synthetic import ar_series
    n, p, cfg, idx, lo, hi = args
    return ar_series(int(n), int(p), config_id=cfg, series_index=idx, root_lo=lo, root_hi=hi).y


def gen_many(shapes, cfg, lo=1.2, hi=3.0):
    """Seeded series for (n, p) shapes, generated in a spawn process pool (before any CUDA call)."""
    import multiprocessing as mp
    jobs = [(n, p, cfg, k, lo, hi) for k, (n, p) in enumerate(shapes)]
    if len(jobs) < 8:
        return [_gen_one(j) for j in jobs]
    with mp.get_context("spawn").Pool(min(16, os.cpu_count() or 1)) as pool:
        return pool.map(_gen_one, jobs, chunksize=4)


def make_series(wl):
    from synthetic import ar_series
    return ar_series(wl["n"], wl["p"], config_id=wl["config_id"], root_lo=wl["root_lo"], root_hi=wl["root_hi"],
                     noise=wl["noise"])


# ---------------------------------------------------------------------------------------------------------
def run_reference(args, wl):
    """The oracle on the host cores, each step a bounded sample of the workload: the first rows of the series."""
    world, rank, _ = dist()
    if rank != 0:
        return
    import numpy as np
    import oracle
    s = make_series(wl)
    p = wl["p"]
    m_full = wl["n"] - p
    m_s = min(m_full, 1 << 19)
    ys = s.y[: m_s + p]
    for _ in range(args.warmup):
        oracle.ols_qr(ys, p)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.ols_qr(ys, p)
    dt = (time.perf_counter() - t0) / args.steps
    per_solve = dt * (m_full / m_s)      # dense QR cost is linear in the row count
    value = 1.0 / per_solve
    sample = f"oracle (blocked Householder QR, float64) on the first {m_s} of {m_full} rows per step; " \
             f"solves/s scaled by {m_full / m_s:.3g}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_solve * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"], "n": wl["n"], "p": p},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------------------
def run_ours(args, wl):
    import numpy as np
    import torch

    import paper_2112_12994_gb300 as tols

    world, rank, local = dist()
    from synthetic import batch_shapes
    batch_in = serve_in = None
    if args.batch_series > 0:
        bn, bp = batch_shapes(args.batch_series, config_id=4, n_lo=1e4, n_hi=1e6, p_lo=5, p_hi=200)
        batch_in = (gen_many(list(zip(bn, bp)), 4), [int(x) for x in bp])
    if args.serve_requests > 0:
        sn, sp = batch_shapes(args.serve_requests, config_id=5, n_lo=1e3, n_hi=1e7, p_lo=1, p_hi=300,
                              p_log_uniform=True)
        serve_in = (gen_many(list(zip(sn, sp)), 5), [int(x) for x in sp])
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ranks = Ranks(world, rank, dev)
    barrier, max_over_ranks = ranks.barrier, ranks.max

    s = make_series(wl)
    n, p, tol = wl["n"], wl["p"], wl["tol"]
    m = n - p
    stream = torch.cuda.Stream(dev)
    d_y = torch.tensor(s.y, dtype=torch.float64, device=dev)
    d_phi = torch.empty(p, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed_solves(ctx, steps, host_y=None, phi_host=None):
        times, infos = [], []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)                       # evict y and the work vectors from L2 (not timed)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if host_y is None:
                _, info, rc = tols.toeplitz_ols_solve_device(ctx, d_y, n, p, d_phi, tol)
            else:
                phi, _, info, rc = tols.toeplitz_ols_solve(ctx, host_y, p, tol)
                phi_host[:] = phi
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        return times, infos

    results = {}
    for name, prec in (("fp64", tols.TOLS_FP64), ("mixed", tols.TOLS_MIXED)):
        ctx = tols.Context(precision=prec, device=local, cuda_stream=stream.cuda_stream)
        timed_solves(ctx, args.warmup)
        tols.toeplitz_ols_profile(ctx, True)
        clocks = ClockSampler(_smi_index(local)) if name == "fp64" else None
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        times, infos = timed_solves(ctx, args.steps)
        torch.cuda.synchronize()
        barrier()
        clk = clocks.stop() if clocks else None
        prof = {tols.PROFILE_CLASS_NAMES[k]: tols.toeplitz_ols_profile_read(ctx, k)
                for k in range(tols.TOLS_PROFILE_CLASSES)}
        launches, _ = tols.toeplitz_ols_profile_read(ctx, -1)
        tols.toeplitz_ols_profile(ctx, False)
        phi = d_phi.cpu().numpy().copy()
        total_ms = max_over_ranks(sum(times))
        results[name] = dict(times=times, infos=infos, prof=prof, launches=launches, phi=phi, total_ms=total_ms,
                             clocks=clk, ctx=ctx)

    # end to end: pinned host series in, phi out, through toeplitz_ols_solve (FP64, the headline precision)
    pinned = torch.empty(n, dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.from_numpy(s.y))
    host_y = pinned.numpy()
    phi_h = np.zeros(p)
    ctx = results["fp64"]["ctx"]
    timed_solves(ctx, 1, host_y, phi_h)
    barrier()
    torch.cuda.synchronize()
    e2e_times, _ = timed_solves(ctx, args.steps, host_y, phi_h)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = max_over_ranks(sum(e2e_times))

    batched = batched_mixed = serving = None
    if batch_in:
        batched = run_batched(tols, torch, dev, stream, batch_in, args, barrier, max_over_ranks, world, tols.TOLS_FP64)
        batched_mixed = run_batched(tols, torch, dev, stream, batch_in, args, barrier, max_over_ranks, world,
                                    tols.TOLS_MIXED)
    if serve_in:
        serving = run_serving(tols, serve_in, args)
    order_sweep = run_order_sweep(tols, torch, s.y, args) if args.pacf_lags > 0 else None
    lsar = (run_lsar(tols, torch, s.y, args, order_sweep["ms_per_sweep"] if order_sweep and
                     order_sweep["lags"] == args.lsar_lags else None) if args.lsar_lags > 0 else None)

    hbm_peak, hbm_src = peaks()
    r64, rmx = results["fp64"], results["mixed"]
    K = args.steps
    value = whole_job_rate(world, K, r64["total_ms"] / 1e3)
    mixed_value = whole_job_rate(world, K, rmx["total_ms"] / 1e3)

    def per_launch(prof, key):
        cnt, ms = prof[key]
        return (ms / cnt if cnt else float("nan")), cnt

    # dominant kernel of the FP64 step and its roofline (float64 FMA units bound it; see the design notes).
    # Flops per launch: direct products 4 m p (2 m p multiply-adds). Overlap-save FFT pass: per tile of
    # L = N - pad16(p + 1) rows one inverse and one forward real N-point transform, 2 x 2.5 N log2 N (the window
    # spectra are formed once per solve, the X^T u spectra are summed per CTA and transformed back once).
    dom = max((k for k in r64["prof"] if r64["prof"][k][0] > 0 and k.startswith("pass_")),
              key=lambda k: r64["prof"][k][1])
    avg_ms, cnt = per_launch(r64["prof"], dom)
    lags = p + 1 if dom.endswith("gram") else p
    fft_used = r64["infos"][-1]["product_used"] == tols.TOLS_PRODUCT_FFT
    if fft_used:
        N = 2048
        pg = ((p + 1 + 15) // 16) * 16
        tiles = math.ceil(m / (N - pg))
        if dom.endswith("gram"):    # one forward transform per tile plus the direct edge corrections
            flops = tiles * (2.5 * N * math.log2(N) + 2.0 * pg * (p + 1))
        else:
            flops = tiles * 5.0 * N * math.log2(N)
        kname = f"fft_pass_kernel<double> ({dom})"
    else:
        flops = (2.0 if dom.endswith("gram") else 4.0) * m * lags
        kname = f"pass_kernel<double> ({dom})"
    achieved_tf = flops / (avg_ms * 1e-3) / 1e12
    byts_fp64 = 8.0 * n + 16.0 * m
    # DRAM traffic of the FFT check/LSQR pass from an ncu capture of the same kernel (n = 2^26, p = 100: 1.106 GB
    # read + 0.508 GB written per launch, 24.05 B per row of y), scaled to this launch's rows
    traffic = 24.05 * n if (fft_used and not dom.endswith("gram") and p == 100) else None
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved_tf,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved_tf / FP64_PEAK_TFLOPS,
                "traffic": traffic, "traffic_source": "ncu dram__bytes_read+write of fft_pass_kernel<double> at "
                                                      "n = 2^26, p = 100, scaled by rows" if traffic else None, "peak_source": "derived: 152 SMs x 4 FP64 flop/clk x 2.07 GHz",
                "flop_per_launch": flops, "avg_launch_ms": avg_ms, "launches": cnt,
                "product": "fft" if fft_used else "direct"}
    mx_dom = "pass_f32_lsqr" if rmx["prof"]["pass_f32_lsqr"][0] else "pass_f32_necorr"
    mx_ms, mx_cnt = per_launch(rmx["prof"], mx_dom)
    byts_mx = 4.0 * n + 8.0 * m
    mx_gbs = byts_mx / (mx_ms * 1e-3) / 1e9 if mx_cnt else None
    fp64_pass_ms, _ = per_launch(r64["prof"], "pass_f64_lsqr")

    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": K,
           "warmup": args.warmup, "ms_per_step": r64["total_ms"] / K, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic: seeded stationary AR series (see config)",
           "config": {"workload": wl["desc"], "n": n, "p": p, "tol": tol, "series_per_rank": 1,
                      "l2": f"flushed between steps ({L2_FLUSH_BYTES >> 20} MiB write, not timed)",
                      "parallelism": "replicas" if world > 1 else "single"},
           "roofline": roofline,
           "matvec": {"fp64_pass_ms": fp64_pass_ms,
                      "fp64_pass_gbs": byts_fp64 / (fp64_pass_ms * 1e-3) / 1e9 if fp64_pass_ms == fp64_pass_ms else None,
                      "mixed_pass_kernel": mx_dom, "mixed_pass_ms": mx_ms, "mixed_pass_gbs": mx_gbs,
                      "mixed_pass_frac_hbm": (mx_gbs / hbm_peak) if mx_gbs else None,
                      "hbm_peak_gbs": hbm_peak, "hbm_peak_source": hbm_src,
                      "bytes_per_pass": {"fp64": byts_fp64, "mixed": byts_mx}},
           "mixed": {"value": mixed_value, "unit": "solves/s", "ms_per_step": rmx["total_ms"] / K,
                     "vs_fp64": mixed_value / value,
                     "precision_used": rmx["infos"][-1]["precision_used"], "iters": rmx["infos"][-1]["iters"],
                     "sweeps": rmx["infos"][-1]["sweeps"], "ne_ratio": rmx["infos"][-1]["ne_ratio"]},
           "latency_ms": {"fp64_p50": float(np.percentile(r64["times"], 50)),
                          "fp64_p99": float(np.percentile(r64["times"], 99)),
                          "mixed_p50": float(np.percentile(rmx["times"], 50)),
                          "mixed_p99": float(np.percentile(rmx["times"], 99))},
           "solve": {"iters": r64["infos"][-1]["iters"], "sweeps": r64["infos"][-1]["sweeps"],
                     "ne_ratio": r64["infos"][-1]["ne_ratio"], "cond_est": r64["infos"][-1]["cond_est"],
                     "status": r64["infos"][-1]["status"]},
           "e2e": {"value": whole_job_rate(world, K, e2e_ms / 1e3), "unit": "solves/s", "h2d_bytes_per_step": 8 * n,
                   "d2h_bytes_per_step": 8 * p},
           "batched": batched,
           "batched_mixed": batched_mixed,
           "serving": serving,
           "order_sweep": order_sweep,
           "lsar": lsar,
           "gpu_launches": int(r64["launches"] + rmx["launches"]),
           "clocks": r64["clocks"],
           "kernel_ms": {k: {"launches": v[0], "total_ms": v[1]} for k, v in r64["prof"].items() if v[0]}}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        solves = 0
        t0 = time.perf_counter()
        while solves < 3 and (solves == 0 or time.perf_counter() - t0 < 10.0):   # about 10-15 s of CPU work
            ref = oracle.ols_qr(s.y, p)
            solves += 1
        dt = (time.perf_counter() - t0) / solves
        out["cpu_baseline"] = {"value": 1.0 / dt, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                               "sample": f"{solves} full solves of the same series (blocked Householder QR, float64)"}
        out["accuracy"] = {"fp64_coef_rel_err": float(np.linalg.norm(r64["phi"] - ref.phi) / np.linalg.norm(ref.phi)),
                           "mixed_coef_rel_err": float(np.linalg.norm(rmx["phi"] - ref.phi) / np.linalg.norm(ref.phi)),
                           "oracle_kappa": ref.kappa, "oracle_forward_bound": ref.forward_error_bound(),
                           "oracle_ne_ratio": ref.ne_ratio}
    for r in results.values():
        r["ctx"].close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    ranks.close()


def run_batched(tols, torch, dev, stream, batch_in, args, barrier, max_over_ranks, world, prec):
    """Many series of uneven length in one batched solve, series resident in HBM."""
    import numpy as np
    ys, ps = batch_in
    d_ys = [torch.tensor(y, dtype=torch.float64, device=dev) for y in ys]
    d_phi = torch.empty(sum(ps), dtype=torch.float64, device=dev)
    steps = max(2, min(args.steps, 5))
    out = {"series": len(ys), "sum_n": int(sum(y.size for y in ys)),
           "precision": "fp64" if prec == tols.TOLS_FP64 else "mixed",
           "workload": "n log-uniform in [1e4, 1e6], p uniform in [5, 200], roots |r| in U[1.2, 3], N(0,1)"}
    with tols.Context(precision=prec, device=dev.index, cuda_stream=stream.cuda_stream) as ctx:
        tols.toeplitz_ols_solve_batched_device(ctx, d_ys, ps, d_phi, BATCH_TOL)       # warm-up
        tols.toeplitz_ols_profile(ctx, True)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(steps):
            rn, infos, rc = tols.toeplitz_ols_solve_batched_device(ctx, d_ys, ps, d_phi, BATCH_TOL)
        torch.cuda.synchronize()
        barrier()
        dt = max_over_ranks(time.perf_counter() - t0)
        launches, _ = tols.toeplitz_ols_profile_read(ctx, -1)
        f32 = tols.toeplitz_ols_profile_read(ctx, 1)
        tols.toeplitz_ols_profile(ctx, False)
        # end to end from host memory through toeplitz_ols_solve_batched
        t1 = time.perf_counter()
        phis_h, _, _, _ = tols.toeplitz_ols_solve_batched(ctx, ys, ps, BATCH_TOL)
        e2e_dt = time.perf_counter() - t1
    status = [i["status"] for i in infos]
    out.update({"value": whole_job_rate(world, len(ys) * steps, dt), "unit": "solves/s", "ms_per_batch": 1e3 * dt / steps,
                "steps": steps, "tol": BATCH_TOL, "statuses_ok": int(sum(1 for x in status if x == 0)),
                "statuses_not_converged": int(sum(1 for x in status if x == 1)),
                "fp64_fallbacks": int(sum(1 for i in infos if i["precision_used"] == 0)),
                "mean_iters": float(np.mean([i["iters"] for i in infos])),
                "max_iters": int(max(i["iters"] for i in infos)),
                "e2e_solves_per_s": len(ys) / e2e_dt, "gpu_launches": int(launches),
                "f32_lsqr_pass_launches": f32[0], "f32_lsqr_pass_ms": f32[1]})
    # accuracy on a few series against the oracle (timed as the CPU baseline of this workload)
    import oracle
    phi_all = d_phi.cpu().numpy()
    offs = np.concatenate([[0], np.cumsum(ps)])
    errs, t_or, rows = [], 0.0, 0
    for k in range(0, len(ys), max(1, len(ys) // 4))[:4]:
        t2 = time.perf_counter()
        ref = oracle.ols_qr(ys[k], ps[k])
        t_or += time.perf_counter() - t2
        rows += 1
        errs.append(float(np.linalg.norm(phi_all[offs[k]:offs[k + 1]] - ref.phi) / np.linalg.norm(ref.phi)))
    out["max_coef_rel_err_sampled"] = max(errs)
    out["cpu_baseline"] = {"value": rows / t_or, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                           "sample": f"{rows} series of the batch"}
    return out


def run_order_sweep(tols, torch, y, args):
    """PACF of the bench series: the fits of order 1 .. h_max as one batch (toeplitz_ols_pacf, host series)."""
    import numpy as np
    h = args.pacf_lags
    with tols.Context(precision=tols.TOLS_FP64) as ctx:
        tols.toeplitz_ols_pacf(ctx, y, h, 1e-10)                      # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tau, order, infos, rc = tols.toeplitz_ols_pacf(ctx, y, h, 1e-10)
        dt = time.perf_counter() - t0
    return {"lags": h, "fits_per_s": h / dt, "ms_per_sweep": dt * 1e3, "order_estimate": order,
            "statuses_ok": int(sum(1 for i in infos if i["status"] == 0)),
            "max_iters": int(max(i["iters"] for i in infos)),
            "workload": "AR(h), h = 1 .. lags, fitted to the bench series (n = 2^22), float64, tol 1e-10, "
                        "end to end from host memory"}


def run_lsar(tols, torch, y, args, exact_ms):
    """Algorithm LSAR on the bench series: compressed fits of lags 1 .. p_bar with c sampled rows each, series and
    uniforms resident on the device (toeplitz_ols_lsar); timed with CUDA events after one warm-up sweep."""
    from synthetic import lsar_uniforms
    p_bar, c = args.lsar_lags, args.lsar_c
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_u = torch.tensor(lsar_uniforms(p_bar, c, config_id=2), dtype=torch.float64, device="cuda")
    times = []
    with tols.Context(precision=tols.TOLS_FP64) as ctx:
        tau, order, _, rc = tols.toeplitz_ols_lsar(ctx, d_y, y.size, p_bar, c, d_u)     # warm-up
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tau, order, _, rc = tols.toeplitz_ols_lsar(ctx, d_y, y.size, p_bar, c, d_u)
            times.append(time.perf_counter() - t0)
    ms = min(times) * 1e3
    res = {"lags": p_bar, "c": c, "ms_per_sweep": ms, "lags_per_s": p_bar / (ms * 1e-3), "order_estimate": order,
           "status": rc, "tau_finite": bool(all(math.isfinite(t) for t in tau)),
           "workload": "Algorithm LSAR on the bench series (n = 2^22): lags 1 .. p_bar on n - p_bar rows, c rows "
                       "sampled per lag, series and uniforms in HBM, best of 3 sweeps (host clock around the call, "
                       "which returns after the device finishes)"}
    if exact_ms:
        res["exact_sweep_ms"] = exact_ms
        res["speedup_vs_exact_sweep"] = exact_ms / ms
    return res


def run_rh(tols, torch, y, args):
    """The Repeated Halving variant of LSAR on the bench series (toeplitz_ols_rh_lsar): halvings down to c rows,
    a k-row sketch per level, then lags 1 .. p_bar; draws and series resident on the device; best of 3."""
    import numpy as np
    from synthetic import lsar_uniforms, rh_draws
    p_bar, c, k = args.lsar_lags, args.lsar_c, args.rh_sketch
    m = y.size - p_bar
    keep, gauss, rh_unif = rh_draws(m, c, k, c, config_id=2)
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_sk = torch.tensor(np.concatenate([g.reshape(-1) for g in gauss]), dtype=torch.float64, device="cuda")
    d_rh = torch.tensor(np.stack(rh_unif), dtype=torch.float64, device="cuda")
    d_u = torch.tensor(lsar_uniforms(p_bar, c, config_id=2), dtype=torch.float64, device="cuda")
    times = []
    with tols.Context(precision=tols.TOLS_FP64) as ctx:
        tau, order, _, rc = tols.toeplitz_ols_rh_lsar(ctx, d_y, y.size, p_bar, c, k, keep, d_sk, d_rh, d_u)
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            tau, order, _, rc = tols.toeplitz_ols_rh_lsar(ctx, d_y, y.size, p_bar, c, k, keep, d_sk, d_rh, d_u)
            times.append(time.perf_counter() - t0)
    ms = min(times) * 1e3
    return {"lags": p_bar, "c": c, "k": k, "levels": len(keep), "ms_per_sweep": ms, "lags_per_s": p_bar / (ms * 1e-3),
            "order_estimate": order, "status": rc, "tau_finite": bool(all(math.isfinite(t) for t in tau)),
            "workload": "Repeated Halving variant of LSAR on the bench series (n = 2^22): halvings to c rows, "
                        "k-row Gaussian sketches, lags 1 .. p_bar with c rows each; inputs in HBM, best of 3 "
                        "(host clock around the call; the halving lists are copied to the device inside it)"}


def run_srht(tols, torch, y, p, args):
    """Algorithm SRHT (toeplitz_ols_srht) for the order-p fit of the bench series: random signs, the normalised
    Hadamard transform of the p+1 padded columns, c sampled rows, the compressed fit; best of 3."""
    import numpy as np
    from synthetic import srht_draws
    c = args.lsar_c
    signs, rows = srht_draws(y.size - p, c, config_id=2)
    d_y = torch.tensor(y, dtype=torch.float64, device="cuda")
    d_s = torch.tensor(signs, dtype=torch.float64, device="cuda")
    d_r = torch.tensor(rows.astype(np.int64), device="cuda")
    d_phi = torch.empty(p, dtype=torch.float64, device="cuda")
    times = []
    with tols.Context(precision=tols.TOLS_FP64) as ctx:
        rc = tols.toeplitz_ols_srht(ctx, d_y, y.size, p, d_s, d_r, d_phi)
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc = tols.toeplitz_ols_srht(ctx, d_y, y.size, p, d_s, d_r, d_phi)
            times.append(time.perf_counter() - t0)
    ms = min(times) * 1e3
    return {"p": p, "c": c, "m2": int(signs.size), "ms_per_fit": ms, "fits_per_s": 1e3 / ms, "status": rc,
            "workload": "Algorithm SRHT for the AR(p) fit of the bench series (n = 2^22): (p+1) columns of "
                        "2^22 padded rows through the Hadamard transform, c rows sampled; best of 3 (host clock)"}


def run_serving(tols, serve_in, args):
    """Continuous batching: saturation throughput, then Poisson arrivals at half of it; p50/p99 latency."""
    import numpy as np
    ys, ps = serve_in
    res = {"requests": len(ys), "sum_n": int(sum(y.size for y in ys)), "precision": "fp64",
           "workload": "n log-uniform in [1e3, 1e7], p log-uniform in [1, 300], roots |r| in U[1.2, 3], N(0,1)"}

    def run(rate):
        rng = np.random.default_rng(5)
        arrivals = np.zeros(len(ys)) if rate is None else np.cumsum(rng.exponential(1.0 / rate, size=len(ys)))
        with tols.Server(precision=tols.TOLS_FP64, burst=4) as srv:
            t0 = time.perf_counter()
            nxt, done, lat = 0, [], []
            while len(done) < len(ys):
                now = time.perf_counter() - t0
                while nxt < len(ys) and arrivals[nxt] <= now:
                    rc = srv.submit(nxt, ys[nxt], ps[nxt], BATCH_TOL)
                    assert rc == 0, rc
                    nxt += 1
                active, queued = srv.step()
                for r in srv.poll():
                    done.append(r)
                if active == 0 and queued == 0 and nxt < len(ys):
                    time.sleep(max(0.0, min(0.01, arrivals[nxt] - (time.perf_counter() - t0))))
            makespan = time.perf_counter() - t0
        lat = np.array([r["latency_s"] for r in done])
        ok = sum(1 for r in done if r["status"] == 0)
        return {"solves_per_s": len(done) / makespan, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3), "makespan_s": makespan, "ok": ok}

    sat = run(None)
    res["saturation"] = sat
    res["poisson_half_rate"] = dict(run(0.5 * sat["solves_per_s"]), rate_per_s=0.5 * sat["solves_per_s"])
    return res


def run_batch_only(args):
    """One float64 batched solve of the batch workload (after one warm-up solve), timed on the host."""
    import numpy as np
    import torch

    import paper_2112_12994_gb300 as tols
    from synthetic import batch_shapes
    bn, bp = batch_shapes(args.batch_series, config_id=4, n_lo=1e4, n_hi=1e6, p_lo=5, p_hi=200)
    ys = gen_many(list(zip(bn, bp)), 4)
    ps = [int(x) for x in bp]
    dev = torch.device("cuda", 0)
    d_ys = [torch.tensor(y, dtype=torch.float64, device=dev) for y in ys]
    d_phi = torch.empty(sum(ps), dtype=torch.float64, device=dev)
    with tols.Context(precision=tols.TOLS_FP64) as ctx:
        tols.toeplitz_ols_solve_batched_device(ctx, d_ys, ps, d_phi, BATCH_TOL)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rn, infos, rc = tols.toeplitz_ols_solve_batched_device(ctx, d_ys, ps, d_phi, BATCH_TOL)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
    it = np.array([i["iters"] for i in infos])
    print(json.dumps({"batch_only": True, "series": len(ys), "sum_n": int(sum(y.size for y in ys)), "seconds": dt,
                      "solves_per_s": len(ys) / dt, "mean_iters": float(it.mean()), "max_iters": int(it.max()),
                      "sampled_qr": int(sum(1 for i in infos if i["precond_used"] == 2))}), flush=True)


def run_kernel_only(args, wl):
    """The fused pass u_new = X v - c u_old, ||u_new||^2, X^T u_new alone, in both precisions."""
    import numpy as np
    import torch

    import paper_2112_12994_gb300 as tols
    if args.p:
        wl = dict(wl, p=args.p)
    s = make_series(wl)
    n, p = wl["n"], wl["p"]
    m = n - p
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(dev)
    rng = np.random.default_rng(1)
    v = torch.tensor(rng.standard_normal(p), dtype=torch.float64, device=dev)
    t = torch.empty(p, dtype=torch.float64, device=dev)
    out = {"kernel_only": True, "workload": wl["desc"], "n": n, "p": p}
    hbm, src = peaks()
    for prod_name, prod in (("direct", tols.TOLS_PRODUCT_DIRECT), ("fft", tols.TOLS_PRODUCT_FFT)):
        with tols.Context(precision=tols.TOLS_FP64, product=prod, cuda_stream=stream.cuda_stream) as ctx:
            for name, dt, prec, nbytes, flops in (("fp64", torch.float64, tols.TOLS_FP64, 8.0 * n + 16.0 * m, 4.0 * m * p),
                                                  ("fp32", torch.float32, tols.TOLS_MIXED, 4.0 * n + 8.0 * m, 4.0 * m * p)):
                if args.only and f"{prod_name}_{name}" not in args.only:
                    continue
                d_y = torch.tensor(s.y, dtype=dt, device=dev)
                u0 = torch.tensor(rng.standard_normal(m), dtype=dt, device=dev)
                u1 = torch.empty(m, dtype=dt, device=dev)
                times = []
                for _ in range(args.reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    tols.toeplitz_ols_gk_pass(ctx, prec, d_y, n, p, v, u0, 0.5, u1, t)
                    e1.record(stream)
                    e1.synchronize()
                    times.append(e0.elapsed_time(e1))
                ms = min(times)
                out[f"{prod_name}_{name}"] = {"ms": ms, "gbs": nbytes / (ms * 1e-3) / 1e9,
                                               "frac_hbm": nbytes / (ms * 1e-3) / 1e9 / hbm,
                                               "tflops_equiv": flops / (ms * 1e-3) / 1e12, "bytes": nbytes}
                del d_y, u0, u1
    out["hbm_peak_gbs"] = hbm
    out["hbm_peak_source"] = src
    print(json.dumps(out), flush=True)


def _smi_index(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    ids = [v for v in vis.split(",") if v.strip()]
    if ids and local < len(ids) and ids[local].strip().isdigit():
        return int(ids[local])
    return local


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
    elif args.kernel_only:
        run_kernel_only(args, wl)
    elif args.batch_only:
        run_batch_only(args)
    elif args.srht_only:
        import torch

        import paper_2112_12994_gb300 as tols
        print(json.dumps({"srht_only": True, **run_srht(tols, torch, make_series(wl).y, wl["p"], args)}), flush=True)
    elif args.rh_only:
        import torch

        import paper_2112_12994_gb300 as tols
        print(json.dumps({"rh_only": True, **run_rh(tols, torch, make_series(wl).y, args)}), flush=True)
    elif args.lsar_only:
        import torch

        import paper_2112_12994_gb300 as tols
        print(json.dumps({"lsar_only": True, **run_lsar(tols, torch, make_series(wl).y, args, None)}), flush=True)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
