"""Benchmark: adaptive KRP TT-rounding throughput on one GB300 (replicas for N > 1).

Workload: the formal sum of 4 scaled copies of a random TT (d=20, n=50, rank 50, entries
N(0,1)/sqrt(n r)) plus rank-10 noise at 1e-7 relative norm: formal rank 210, 318 MB of FP64
cores (larger than the 129 MB L2, so no flush is needed between steps).  One step = one
adaptive rounding (Algorithm 6) to tol 1e-6 with block size 10 and the exact input norm,
cores resident in HBM; the headline step rounds it on --streams (default 3) CUDA streams at once,
one host thread each, every block loop on its share of the SMs (p50/p99 are per-rounding
latencies under that load; the one-at-a-time figures are in `single_stream`).  Reported beside
it: the deterministic FP64
TT-rounding (Algorithm 1) on the same GPU, the end-to-end rate through host buffers, the
roofline of the dominant kernel (the adaptive block loop of Algorithm 6, FP64 arithmetic) and of
the tensor-core partial contractions (Algorithm 3, HBM), both timed by the library's CUDA events
inside the timed region, and the CPU oracle on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--precision fp64|sliced]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

TOL, BLOCK, SEED = 1e-6, 10, 2024
METRIC = "TT roundings/sec (adaptive KRP, tol 1e-6) with p50/p99 ms vs FP64 deterministic rounding"


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    def __init__(self):
        self.samples, self._p, self._t = [], None, None

    def start(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", os.environ.get("LOCAL_RANK", "0"), f"--query-gpu={q}",
                                        "--format=csv,noheader,nounits", "-lms", "200"],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self._p = None
            return
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()

    def _read(self):
        for line in self._p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self._p:
            self._p.terminate()
            try:
                self._p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self._p.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples for i in range(4) if "Active" in s[3 + i]
                          and "Not" not in s[3 + i]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# FP64 peak from unit counts and clocks: 152 SMs x 2 FP64 FMA per clock x 2 flop x 2.07 GHz (the
# fallback when the GEMM probe below cannot run)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def probe_peaks() -> dict:
    """Measured FP64 and TF32 GEMM rates of this GPU (torch.matmul, i.e. cuBLAS, 8192^3 FP64 and
    FP32-with-TF32, best of 3 after one warm-up; CUDA events): the denominators of the FP64-pipe
    roofline, beside the measured HBM and BF16 figures."""
    import torch
    out = {}
    old = torch.backends.cuda.matmul.allow_tf32
    try:
        for name, dt, tf32 in (("fp64_tflops", torch.float64, False), ("tf32_tflops", torch.float32, True)):
            torch.backends.cuda.matmul.allow_tf32 = tf32
            n = 8192
            a = torch.randn(n, n, dtype=dt, device="cuda")
            b = torch.randn(n, n, dtype=dt, device="cuda")
            torch.matmul(a, b)
            best = float("inf")
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * n ** 3 / (best / 1e3) / 1e12
            del a, b
    finally:
        torch.backends.cuda.matmul.allow_tf32 = old
    out["how"] = "torch.matmul 8192^3 (cuBLAS), best of 3 after a warm-up, CUDA events"
    return out

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# this workload in sliced precision, for the kernels as they stand (the capture command is in
# profiles/): the FP64 block loop's figure is the median over full-rank cores, the partial
# contraction's the mean over all 18 launches of one pass.  Other precisions run other kernels.
TRAFFIC_SLICED = {"block_loop": 2.454e6, "rl_kernel": 17.98e6}


def serving_run(B, nreq: int, workers: int, budget: int, nreq_open: int | None = None) -> dict:
    """The serving stream (Poisson arrivals, mean gap 2 ms; each request a sum of 2-6 random TTs
    with d 8-32, n 16-128, ranks 20-100, tol 1e-4/1e-6/1e-8): its first `nreq` requests (closed
    loop) and its first `nreq_open` (open loop; default `nreq`), given to
    the library's request server as summands in host memory.  A producer generates the requests
    (on a pool of host threads, each request from a generator of its own) while the server works,
    holding at most a window of them (the whole stream's summands are ~80 GB); each request's host
    data is dropped once its result is collected.  Closed loop: a
    request is submitted as soon as it is generated and the window has room (throughput).  Open loop:
    each is submitted at its arrival time, or when generated if that is later (latency under that
    load; the stream arrives ~100 times faster than one GPU rounds it, so queueing dominates)."""
    import collections
    import queue
    from concurrent.futures import ThreadPoolExecutor

    import workloads as WL
    window = max(4, 3 * workers)
    gen_threads = max(1, min(8, (os.cpu_count() or 4) // 2))
    srv = B.Server(workers=workers, device_budget=budget)
    opts = B.options(precision=B.TTR_PREC_SLICED)

    def producer(q, stop, pool, count):
        for spec in WL.c4_specs(count=count):
            fut = pool.submit(WL.c4_request, spec, 4, False)
            while not stop.is_set():
                try:
                    q.put(fut, timeout=0.5)
                    break
                except queue.Full:
                    continue
            if stop.is_set():
                return
        q.put(None)

    try:
        # warm-up: one small request (kernel attributes, memory pool)
        small = next(WL.c4_stream(count=512, formal=False, max_bytes=1e8))
        srv.wait(srv.submit(small.tt.summands, small.tol, 0, 7, opts), fetch=False)
        out = {}
        counts = {"closed_loop": nreq, "open_loop": nreq if nreq_open is None else nreq_open}
        for mode in ("closed_loop", "open_loop"):
            if counts[mode] <= 0:
                continue
            q, stop = queue.Queue(maxsize=window), threading.Event()
            pool = ThreadPoolExecutor(max_workers=gen_threads)
            th = threading.Thread(target=producer, args=(q, stop, pool, counts[mode]), daemon=True)
            th.start()
            pending = collections.deque()
            lat, late, ranks_max, formal, inbytes, count = [], [], 0, 0, 0, 0
            t0 = time.perf_counter()

            def collect_one():
                nonlocal ranks_max
                rid = pending.popleft()
                _, info = srv.wait(rid, fetch=False)   # result already in host memory (the worker's D2H)
                lat.append(info["ms_queue"] + info["ms_run"])
                ranks_max = max(ranks_max, max(info["ranks"]))
            try:
                while True:
                    fut = q.get()
                    if fut is None:
                        break
                    r = fut.result()
                    if mode == "open_loop":
                        delay = r.arrival_ms / 1e3 - (time.perf_counter() - t0)
                        if delay > 0:
                            time.sleep(delay)
                        else:
                            late.append(-delay * 1e3)
                    while len(pending) >= window:
                        collect_one()
                    pending.append(srv.submit(r.tt.summands, r.tol, 0, 1000 + r.rid, opts))
                    formal += r.tt.meta["formal_bytes"]
                    inbytes += sum(c.nbytes for x in r.tt.summands for c in x)
                    count += 1
                while pending:
                    collect_one()
            finally:
                stop.set()
                pool.shutdown(wait=True, cancel_futures=True)
            span = time.perf_counter() - t0
            st = srv.stats()
            out[mode] = {"roundings_per_s": count / span, "p50_ms": float(np.percentile(lat, 50)),
                         "p99_ms": float(np.percentile(lat, 99)), "span_s": span, "requests": count,
                         "peak_device_bytes_admitted": int(st["peak_in_use"]), "max_output_rank": ranks_max,
                         "formal_bytes_total": int(formal), "input_bytes_total": int(inbytes)}
            if mode == "open_loop":
                out[mode]["submitted_after_arrival_p50_ms"] = float(np.percentile(late, 50)) if late else 0.0
        out.update({"requests": counts, "workers": workers, "device_budget": budget, "window": window,
                    "generator_threads": gen_threads,
                    "precision": "sliced, slices from each request's tol", "block": "appendix rule (block 0)",
                    "note": "requests of the seeded serving stream (seed 4), generated on host threads while the "
                            "server works, summands in pageable host memory; latency = submit to result in host "
                            "memory (queueing + H2D + rounding + D2H)"})
        return out
    finally:
        srv.close()


def sum_round_run(B, x, opts, args, world, stream, barrier, single, out_ranks) -> dict:
    """The workload as its summands, rounded without forming the formal sum (Remark 3.3, Appendix D):
    one at a time on one stream, CUDA events around each call as in `single_stream`."""
    import torch
    dev_of = {}
    summands = [[dev_of.setdefault(id(c), torch.from_numpy(np.ascontiguousarray(c)).to("cuda")) for c in part]
                for part in x.summands]
    for _ in range(args.warmup):
        with B.round_adaptive_sum(summands, TOL, BLOCK, SEED, opts) as y:
            sum_ranks = y.ranks
    sum_steps = max(3, min(args.steps, 100))
    topts = B.options(precision=opts.precision, nrmx=opts.nrmx, kernel_timing=True)
    kt = {"ms_block_loop": 0.0, "ms_rl_kernel": 0.0, "bytes_rl_kernel": 0.0, "n_rl_kernel": 0}
    barrier()
    sev = [torch.cuda.Event(enable_timing=True) for _ in range(sum_steps + 1)]
    sev[0].record(stream)
    for i in range(sum_steps):
        y = B.round_adaptive_sum(summands, TOL, BLOCK, SEED, topts)
        sum_ranks = y.ranks
        res = y.result
        for key in kt:
            kt[key] += getattr(res, key)
        y.free()
        sev[i + 1].record(stream)
    barrier()
    sum_step_ms = [sev[i].elapsed_time(sev[i + 1]) for i in range(sum_steps)]
    sum_ms = max_over_ranks(sev[0].elapsed_time(sev[-1]), world, "cuda")
    sum_round = {"roundings_per_s": job_rate(sum_steps, world, sum_ms), "ms_per_rounding": sum_ms / sum_steps,
                 "p50_ms": float(np.percentile(sum_step_ms, 50)), "p99_ms": float(np.percentile(sum_step_ms, 99)),
                 "steps": sum_steps, "summands": len(summands), "ranks_out": sum_ranks,
                 "ranks_equal_formal": sum_ranks == out_ranks,
                 "speedup_over_formal_single_stream": single["ms_per_rounding"] / (sum_ms / sum_steps),
                 "share_of_step": {"block_loop": kt["ms_block_loop"] / max(sum_ms, 1e-9),
                                   "partial_contractions": kt["ms_rl_kernel"] / max(sum_ms, 1e-9)},
                 "partial_contractions": None if not kt["n_rl_kernel"] else {
                     "kernel": "grouped partial contractions (one launch per core for all summands)",
                     "ms_per_launch": kt["ms_rl_kernel"] / kt["n_rl_kernel"],
                     "achieved_gbs": kt["bytes_rl_kernel"] / (kt["ms_rl_kernel"] / 1e3) / 1e9,
                     "bytes_per_launch": kt["bytes_rl_kernel"] / kt["n_rl_kernel"],
                     "hbm_frac": kt["bytes_rl_kernel"] / (kt["ms_rl_kernel"] / 1e3) / 1e9 / peaks()[0]["hbm_gbs"]},
                 "note": "tt_round_adaptive_sum on the 4 scaled copies + noise TT (copies share their cores after the "
                         "first), one stream; compare with single_stream, the formal sum of the same input"}
    return sum_round


def e2e_server_run(B, host, opts, workers: int, steps: int):
    """End to end through the library's request server: `steps` requests of the workload, its cores
    in pinned host memory, `workers` in flight; each request is copied to the device, rounded and
    its result copied back to host memory.  Returns (roundings/s, result bytes, steps)."""
    arrays = [h.numpy() for h in host]                       # views of the pinned buffers
    with B.Server(workers=workers, device_budget=64 << 30) as srv:
        srv.wait(srv.submit([arrays], TOL, BLOCK, SEED, opts), fetch=False)   # warm-up
        t0 = time.perf_counter()
        ids = [srv.submit([arrays], TOL, BLOCK, SEED, opts) for _ in range(steps)]
        d2h = 0
        for rid in ids:
            _, info = srv.wait(rid, fetch=False)   # the worker has copied the result to host memory
            d2h = info["result_bytes"]
        dt = time.perf_counter() - t0
    return steps / dt, d2h, steps


def configs_table(B, reps: int) -> dict:
    """Per-configuration timings (the CPU-baseline plan's table): for C1, C2, C3 the GPU
    deterministic FP64 rounding, the GPU KRP rounding in FP64 and sliced form, the oracle's
    deterministic and KRP roundings on the host cores, and the sliced result's distance to the
    oracle's; for C5 (d=50, n=100, formal rank 810, through the sum entry point: its formal sum is
    25 GB) the GPU KRP roundings and the sliced result's error from FP64 inner products.  GPU times
    are CUDA-event medians over `reps` calls, host times wall-clock medians."""
    import torch
    import workloads as WL
    from oracle import rounding as OR
    from oracle import tt as OT

    def gpu_ms(fn, n):
        # one untimed call, then n timed ones; the last result is copied to the host after its timing
        st = torch.cuda.current_stream()
        ts, ranks, res = [], None, None
        for i in range(n + 1):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            y = fn()
            b.record(st)
            torch.cuda.synchronize()
            ranks = y.ranks
            if i == n:
                res = y.to_numpy()
            y.free()
            if i > 0:
                ts.append(a.elapsed_time(b))
        return float(np.median(ts)), ranks, res

    def cpu_ms(fn, n):
        ts, out = [], None
        for _ in range(n):
            t0 = time.perf_counter()
            out = fn()
            ts.append(1e3 * (time.perf_counter() - t0))
        return float(np.median(ts)), out

    rows = []
    for name, x, tol, mode, block in (("c1", WL.c1(), 1e-6, "fixed", 0), ("c2", WL.c2(), 1e-6, "adaptive", 10),
                                      ("c3", WL.c3(), 1e-8, "adaptive", 0)):
        # the operator-applied vector runs with the estimator reading R16 (10 columns, stop at tau / 10)
        est = dict(est_min=10, est_safety=10.0) if name == "c3" else {}
        sl, fp = B.options(precision=B.TTR_PREC_SLICED, **est), B.options(precision=B.TTR_PREC_FP64, **est)
        cores = [torch.from_numpy(c).to("cuda") for c in x.cores]
        for o in (sl, fp):
            o.nrmx = x.norm
        if mode == "fixed":       # fixed rank 8 from a sketch of 13 (oversampling 5)
            krp = lambda o: (lambda: B.round_fixed(cores, 13, SEED, target=8, opts=o))
            oracle_krp = lambda: OR.svd_pass_rl(OR.tt_round_fixed(x.cores, 13, SEED)[0], max_rank=8)
        else:
            krp = lambda o: (lambda: B.round_adaptive(cores, tol, block, SEED, o))
            oracle_krp = lambda: OR.tt_round_adaptive(x.cores, tol, SEED, block=block, nrmx=x.norm, **est)[0]
        det_n = 2 if name == "c2" else reps
        g_det, det_ranks, _ = gpu_ms(lambda: B.round_deterministic(cores, tol), det_n)
        g_fp, fp_ranks, y_fp = gpu_ms(krp(fp), reps)
        g_sl, sl_ranks, y_sl = gpu_ms(krp(sl), max(reps, 20))
        c_det, _ = cpu_ms(lambda: OR.tt_round_deterministic(x.cores, tol), 3)
        c_krp, y_or = cpu_ms(oracle_krp, 5)
        row = {"config": name, "mode": mode, "tol": tol, "cpu_cores": host_cores(),
               "oracle_det_ms": c_det, "oracle_krp_ms": c_krp, "gpu_det_fp64_ms": g_det,
               "gpu_krp_fp64_ms": g_fp, "gpu_krp_sliced_ms": g_sl, "ranks_krp": sl_ranks,
               "ranks_equal_fp64": sl_ranks == fp_ranks, "ranks_det": det_ranks,
               "err_sliced_vs_oracle": OT.tt_dist(y_sl, y_or) / OT.tt_norm(y_or),
               "err_fp64_vs_oracle": OT.tt_dist(y_fp, y_or) / OT.tt_norm(y_or),
               "rel_err_sliced_vs_x": OT.tt_dist(y_sl, x.cores) / x.norm,
               "estimator": "R16 (est_min 10, est_safety 10)" if est else "Algorithm 6 as printed"}
        if name == "c3":
            # the same rounding from the operator and the vector, y never formed in the right-to-left pass
            op, xv = WL.c3_factors()
            opd = [torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in op]
            xvd = [torch.from_numpy(np.ascontiguousarray(c)).to("cuda") for c in xv]
            g_mv, mv_ranks, y_mv = gpu_ms(lambda: B.round_adaptive_matvec(opd, xvd, tol, block, SEED, sl), reps)
            row.update({"gpu_krp_sliced_matvec_fused_ms": g_mv, "ranks_matvec_equal": mv_ranks == sl_ranks,
                        "err_matvec_vs_oracle": OT.tt_dist(y_mv, y_or) / OT.tt_norm(y_or)})
        rows.append(row)
        del cores
    x = WL.c5(formal=False)
    cache = {}
    summ = [[cache.setdefault(id(c), torch.from_numpy(np.ascontiguousarray(c)).to("cuda")) for c in part]
            for part in x.summands]
    sl.nrmx = fp.nrmx = x.norm
    g_sl, sl_ranks, _ = gpu_ms(lambda: B.round_adaptive_sum(summ, 1e-6, 0, SEED, sl), 2)
    g_fp, fp_ranks, _ = gpu_ms(lambda: B.round_adaptive_sum(summ, 1e-6, 0, SEED, fp), 1)
    y = B.round_adaptive_sum(summ, 1e-6, 0, SEED, sl)
    Y = y.to_torch()
    y.free()

    copies = [p for p in summ if p[1].data_ptr() == summ[0][1].data_ptr()]
    others = [p for p in summ if p[1].data_ptr() != summ[0][1].data_ptr()]
    merged = [sum(p[0] for p in copies)] + list(copies[0][1:])
    # X - Y = s T + N - Y (the copies share T's cores after the first, so their first cores add up)
    err = tt_sum_norm([merged] + others + [[-Y[0]] + list(Y[1:])]) / x.norm
    rows.append({"config": "c5", "mode": "adaptive, sum of 5 TTs (formal sum not formed)", "tol": 1e-6,
                 "gpu_krp_fp64_ms": g_fp, "gpu_krp_sliced_ms": g_sl, "ranks_krp_middle": sl_ranks[len(sl_ranks) // 2],
                 "ranks_equal_fp64": sl_ranks == fp_ranks, "err_sliced_vs_x": err,
                 "note": "no oracle or deterministic columns: the formal sum is 25 GB"})
    return {"configs": rows, "oracle_single_thread": oracle_single_thread()}


def oracle_single_thread() -> dict:
    """The oracle's times for C1-C3 with one BLAS thread (a child process: the thread count of the
    BLAS is fixed when NumPy loads), median of 3 after a warm-up."""
    code = r'''
import json, time, numpy as np, workloads as WL
from oracle import rounding as R
out = {}
for name, x, tol, mode, block, est in (("c1", WL.c1(), 1e-6, "fixed", 0, {}), ("c2", WL.c2(), 1e-6, "adaptive", 10, {}),
                                        ("c3", WL.c3(), 1e-8, "adaptive", 0, {"est_min": 10, "est_safety": 10.0})):
    def krp():
        if mode == "fixed":
            return R.svd_pass_rl(R.tt_round_fixed(x.cores, 13, 2024)[0], max_rank=8)
        return R.tt_round_adaptive(x.cores, tol, 2024, block=block, nrmx=x.norm, **est)
    det = lambda: R.tt_round_deterministic(x.cores, tol)
    row = {}
    for key, fn in (("det_ms", det), ("krp_ms", krp)):
        fn()
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            fn()
            ts.append(1e3 * (time.perf_counter() - t0))
        row[key] = float(np.median(ts))
    out[name] = row
print(json.dumps(out))
'''
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1")
    try:
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=600)
        if r.returncode != 0:
            return {"error": r.stderr.strip().splitlines()[-1] if r.stderr.strip() else f"exit {r.returncode}"}
        return {"threads": 1, **json.loads(r.stdout.strip().splitlines()[-1])}
    except Exception as e:  # noqa: BLE001 - reported in the table
        return {"error": f"{type(e).__name__}: {e}"}


def tt_sum_norm(terms) -> float:
    """||sum of the TTs in `terms`|| (lists of torch cores on one device), by left-orthogonalizing
    the block cores of the formal sum with QR, one core at a time: the norm is that of the last
    core after the triangular factors are carried into it.  Unlike an expansion into inner
    products, this resolves a small difference of nearly equal TTs (relative to their norms) to
    FP64 accuracy.  Measurement helper (not the library's path)."""
    import torch
    R = None
    d = len(terms[0])
    for k in range(d):
        blocks = [t[k] for t in terms]
        if k == 0:
            Z = torch.cat(blocks, dim=2)
        elif k == d - 1:
            Z = torch.cat(blocks, dim=0)
        else:
            r0, r1 = sum(b.shape[0] for b in blocks), sum(b.shape[2] for b in blocks)
            Z = torch.zeros((r0, blocks[0].shape[1], r1), dtype=blocks[0].dtype, device=blocks[0].device)
            a = c = 0
            for b in blocks:
                Z[a:a + b.shape[0], :, c:c + b.shape[2]] = b
                a, c = a + b.shape[0], c + b.shape[2]
        if R is not None:
            Z = torch.tensordot(R, Z, dims=([1], [0]))
        if k == d - 1:
            return float(torch.linalg.norm(Z))
        M = Z.reshape(-1, Z.shape[2])
        R = torch.linalg.qr(M, mode="r")[1] if M.shape[0] >= M.shape[1] else M
    return 0.0


def max_over_ranks(ms: float, world: int, device) -> float:
    """The job's time: the largest of the ranks' timed regions (all_reduce MAX when world > 1)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(steps: int, world: int, job_ms: float) -> float:
    """Whole-job throughput: every rank rounds `steps` tensors (replicas, weak scaling)."""
    return world * steps / (job_ms / 1e3)


def concurrent_timed(B, cores, opts_kw, streams: int, rounds: int, share: int = 0) -> dict:
    """`streams` host threads, each on its own CUDA stream with 1/streams of the SMs for the block
    loop, round the same resident input `rounds` times each (one step = one round of every
    stream).  The span is taken with CUDA events: a reference event on the current stream after a
    device synchronisation, and an end event on every worker stream; latency is per call."""
    import threading

    import torch
    nsm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    share = share if share > 0 else max(1, nsm // streams)
    lat = [[] for _ in range(streams)]
    ends = [None] * streams
    launches = [0] * streams
    errs = []
    ready = threading.Barrier(streams + 1)
    go = threading.Event()

    def run(i):
        try:
            s = torch.cuda.Stream()
            opts = B.options(max_sms=share, **opts_kw)
            with torch.cuda.stream(s):
                B.round_adaptive(cores, TOL, BLOCK, SEED, opts, stream=s).free()      # warm-up on this stream
                s.synchronize()
                ready.wait()
                go.wait()
                for _ in range(rounds):
                    t0 = time.perf_counter()
                    y = B.round_adaptive(cores, TOL, BLOCK, SEED, opts, stream=s)
                    launches[i] += y.result.kernel_launches
                    y.free()
                    lat[i].append(1e3 * (time.perf_counter() - t0))
                ends[i] = torch.cuda.Event(enable_timing=True)
                ends[i].record(s)
        except Exception as e:
            errs.append(repr(e))
            ready.abort()

    threads = [threading.Thread(target=run, args=(i,)) for i in range(streams)]
    for t in threads:
        t.start()
    try:
        ready.wait()
    except threading.BrokenBarrierError:
        pass
    torch.cuda.synchronize()
    ref = torch.cuda.Event(enable_timing=True)
    ref.record(torch.cuda.current_stream())
    go.set()
    for t in threads:
        t.join()
    torch.cuda.synchronize()
    if errs:
        raise RuntimeError(errs[0])
    span = max(ref.elapsed_time(e) for e in ends)
    all_lat = [v for l in lat for v in l]
    return {"span_ms": span, "latencies_ms": all_lat, "launches": sum(launches), "max_sms_per_stream": share}


def torch_deterministic(cores, tol):
    """Comparison only (not this library's path): Algorithm 1 with torch's FP64 GPU QR and SVD
    (cuSOLVER), for the speed of a tuned library deterministic TT-rounding on the same GPU."""
    import math

    import torch
    d = len(cores)
    Y = [c.clone() for c in cores]
    for k in range(d - 1, 0, -1):                                 # right-to-left orthogonalization
        r0, n, r1 = Y[k].shape
        Q, R = torch.linalg.qr(Y[k].reshape(r0, n * r1).T)
        rk = Q.shape[1]
        Y[k] = Q.T.reshape(rk, n, r1)
        Y[k - 1] = (Y[k - 1].reshape(-1, r0) @ R.T).reshape(Y[k - 1].shape[0], Y[k - 1].shape[1], rk)
    tau = float(torch.linalg.norm(Y[0])) * tol / math.sqrt(d - 1)
    ranks = [1]
    for k in range(d - 1):
        r0, n, r1 = Y[k].shape
        Q, R = torch.linalg.qr(Y[k].reshape(r0 * n, r1))
        U, sv, Vt = torch.linalg.svd(R, full_matrices=False)
        tail = torch.sqrt(torch.flip(torch.cumsum(torch.flip(sv * sv, [0]), 0), [0]))
        keep = int((tail > tau).sum().item())
        rp = max(1, keep)
        Y[k] = (Q @ U[:, :rp]).reshape(r0, n, rp)
        q0, qn, q1 = Y[k + 1].shape
        Y[k + 1] = ((sv[:rp, None] * Vt[:rp]) @ Y[k + 1].reshape(q0, qn * q1)).reshape(rp, qn, q1)
        ranks.append(rp)
    ranks.append(1)
    return ranks


def cpu_oracle_rate(x, budget_s=15.0):
    """The oracle as it stands, on a bounded sample: whole adaptive roundings of the same input."""
    from oracle import rounding as R
    t0, n = time.perf_counter(), 0
    while True:
        R.tt_round_adaptive(x.cores, TOL, SEED, block=BLOCK, nrmx=x.norm)
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 50:
            break
    dt = time.perf_counter() - t0
    return n / dt, n, dt


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def run_reference(args, x):
    """--impl reference: the CPU oracle timed as it stands (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import rounding as R
    for _ in range(args.warmup):
        R.tt_round_adaptive(x.cores, TOL, SEED, block=BLOCK, nrmx=x.norm)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        R.tt_round_adaptive(x.cores, TOL, SEED, block=BLOCK, nrmx=x.norm)
        times.append(time.perf_counter() - t0)
    v = len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "roundings/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
            "p50_ms": 1e3 * float(np.percentile(times, 50)), "p99_ms": 1e3 * float(np.percentile(times, 99)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(x, args.streams),
            "cpu_baseline": {"value": v, "unit": "roundings/s", "cores": host_cores(), "kind": "oracle",
                             "sample": f"{len(times)} whole adaptive roundings of the workload (numpy FP64)"},
            "e2e": {"value": v, "unit": "roundings/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def config(x, streams):
    return {"workload": "c2: 4 x random TT (d=20, n=50, r=50) + rank-10 noise @1e-7, formal rank 210, "
                        "adaptive tol 1e-6, block 10, exact norm", "d": x.d, "n": 50, "formal_rank": 210,
            "tol": TOL, "block": BLOCK, "bytes": x.nbytes, "l2": "inputs (318 MB) larger than L2, no flush",
            "global_batch": streams,
            "batch": f"one step = {streams} roundings in flight at once, one CUDA stream and host thread each, "
                     f"each block loop on 1/{streams} of the SMs"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="sliced", choices=["fp64", "sliced"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--det-steps", type=int, default=2)
    ap.add_argument("--streams", type=int, default=3, help="roundings in flight at once (one stream each)")
    ap.add_argument("--only-main", action="store_true", help="timed rounding loop only (for profiler runs)")
    ap.add_argument("--max-sms", type=int, default=0,
                    help="SMs of each in-flight rounding's block loop (0: SMs / streams)")
    ap.add_argument("--configs", action="store_true",
                    help="print the per-configuration table (GPU and oracle times) instead of the bench line")
    ap.add_argument("--serve-requests", type=int, default=24,
                    help="requests of the serving stream in the closed-loop run (0: skip)")
    ap.add_argument("--serve-open-requests", type=int, default=512,
                    help="requests of the serving stream in the open-loop run at their arrival times "
                         "(512: the whole configured stream; 0: skip)")
    args = ap.parse_args()

    import workloads as WL
    x = WL.c2()
    if args.impl == "reference":
        run_reference(args, x)
        return

    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2511_03598_gb300 import binding as B
    B.lib()
    if args.configs:
        if rank == 0:
            print(json.dumps(configs_table(B, 5)), flush=True)
        return
    prec = B.TTR_PREC_SLICED if args.precision == "sliced" else B.TTR_PREC_FP64
    opts = B.options(precision=prec, nrmx=x.norm)
    topts = B.options(precision=prec, nrmx=x.norm, kernel_timing=True)
    stream = torch.cuda.current_stream()
    cores = [torch.from_numpy(c).to("cuda") for c in x.cores]
    ranks_in = x.ranks
    modes = x.modes

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- warm-up, then the single-stream part: one rounding at a time (kernel events for the rooflines)
    for _ in range(args.warmup):
        with B.round_adaptive(cores, TOL, BLOCK, SEED, opts) as y:
            out_ranks, info = y.ranks, y.info
    clk = ClockSampler()
    clk.start()
    barrier()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    kt = {"ms_block_loop": 0.0, "flops_block_loop": 0.0, "n_block_loop": 0, "ms_rl_kernel": 0.0,
          "bytes_rl_kernel": 0.0, "n_rl_kernel": 0}
    ev[0].record(stream)
    for i in range(args.steps):
        y = B.round_adaptive(cores, TOL, BLOCK, SEED, topts)
        res = y.result                           # the C struct: no per-step Python lists
        for key in kt:
            kt[key] += getattr(res, key)
        y.free()
        ev[i + 1].record(stream)
    barrier()
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    single_total = ev[0].elapsed_time(ev[-1])
    single_ms = max_over_ranks(single_total, world, "cuda")
    single = {"roundings_per_s": job_rate(args.steps, world, single_ms), "ms_per_rounding": single_ms / args.steps,
              "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99))}

    # ---- the timed batch: every step rounds the input on each of STREAMS streams at once
    barrier()
    conc = concurrent_timed(B, cores, {"precision": prec, "nrmx": x.norm}, args.streams, args.steps, args.max_sms)
    barrier()
    clk.stop()
    total_ms = max_over_ranks(conc["span_ms"], world, "cuda")
    value = job_rate(args.steps * args.streams, world, total_ms)
    launches = conc["launches"]
    lat = conc["latencies_ms"]

    if args.only_main:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": "roundings/s", "ms_per_step": total_ms / args.steps,
                              "gpu_launches": int(launches), "only_main": True}), flush=True)
        return
    # ---- rooflines from the library's CUDA events around each launch in the timed region
    w = int(info["width"])
    pk, pk_kind = peaks()
    try:
        probed = probe_peaks()
    except Exception as e:  # noqa: BLE001 - fall back to the derived FP64 peak, and say so
        probed = {"error": f"{type(e).__name__}: {e}"}
    fp64_peak = probed.get("fp64_tflops") or FP64_PEAK_TFLOPS
    fp64_src = ("measured FP64 GEMM (torch.matmul 8192^3, cuBLAS) on this GPU" if "fp64_tflops" in probed else
                "derived from unit counts and clocks: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz")
    traffic = TRAFFIC_SLICED if args.precision == "sliced" else {}
    roof_bl = None
    if kt["n_block_loop"]:
        ach = kt["flops_block_loop"] / (kt["ms_block_loop"] / 1e3) / 1e12
        roof_bl = {"bound": "alu", "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s",
                   "frac": ach / fp64_peak, "traffic": traffic.get("block_loop"),
                   "kernel": "adaptive block loop (Algorithm 6): persistent cooperative FP64 kernel, one launch per core",
                   "peak_source": fp64_src,
                   "per_unit": f"{kt['flops_block_loop'] / kt['n_block_loop']:.3e} FP64 flop per launch (one core's "
                               "blocks: residual projections, Gram matrices, CholeskyQR2, block Gram-Schmidt)",
                   "ms_per_launch": kt["ms_block_loop"] / kt["n_block_loop"],
                   "measured": "single-stream part of the timed run (kernel alone on the GPU)",
                   "share_of_step": kt["ms_block_loop"] / single_total}
    roof_rl = None
    if kt["n_rl_kernel"]:
        ach = kt["bytes_rl_kernel"] / (kt["ms_rl_kernel"] / 1e3) / 1e9
        roof_rl = {"bound": "hbm", "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                   "traffic": traffic.get("rl_kernel"), "kernel": "partial contractions (Algorithm 3): sliced FP64 on BF16 tcgen05, one launch per core",
                   "peak_source": f"hbm_gbs {pk_kind}",
                   "per_unit": f"{kt['bytes_rl_kernel'] / kt['n_rl_kernel']:.3e} B per launch (core read once, "
                               "W_k+1 read, W_k written)",
                   "ms_per_launch": kt["ms_rl_kernel"] / kt["n_rl_kernel"],
                   "measured": "single-stream part of the timed run (kernel alone on the GPU)",
                   "share_of_step": kt["ms_rl_kernel"] / single_total}
        if args.precision == "sliced" and pk.get("bf16_tflops"):
            # the same launches against the tensor pipe: the BF16 MMA work the sliced products issue
            # (s(s+1)/2 digit products of 128 x tn x K_pad per 128-row tile, K padded to chunks of 32)
            s_sl = min(8, max(4, math.ceil((-math.log2(TOL) + 16) / 7)))
            tw = (512 // s_sl) // 16 * 16
            nch = -(-w // tw)
            per = -(-w // nch)
            tn = min(tw, max(16, -(-per // 16) * 16))
            g = 128 // x.modes[0]
            mma = 0.0
            for k in range(2, x.d):                       # the RL launches: W_k for k = d-1 .. 2
                r0, r1 = x.ranks[k - 1], x.ranks[k]
                tiles = -(-r0 // g) * nch
                mma += 2.0 * 128 * tn * (-(-r1 // 32) * 32) * (s_sl * (s_sl + 1) // 2) * tiles
            per_launch = mma / (x.d - 2)
            tach = per_launch / (kt["ms_rl_kernel"] / kt["n_rl_kernel"] / 1e3) / 1e12
            roof_rl["tensor_pipe"] = {"achieved": tach, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
                                      "frac": tach / pk["bf16_tflops"],
                                      "per_unit": f"{per_launch:.3e} BF16 MMA flop per launch ({s_sl} slices: "
                                                  f"{s_sl * (s_sl + 1) // 2} digit products, tile width {tn})",
                                      "peak_source": f"bf16_tflops {pk_kind}"}
    cand = [r for r in (roof_bl, roof_rl) if r]
    roof = max(cand, key=lambda r: r["share_of_step"]) if cand else None
    roof_other = [r for r in cand if r is not roof]

    # ---- the same input as its summands, rounded without forming the formal sum (Remark 3.3,
    # Appendix D), and the serving stream through the library's request server.  Both are reported
    # beside the headline; a failure in either is recorded in its object, not raised.
    try:
        sum_round = sum_round_run(B, x, opts, args, world, stream, barrier, single, out_ranks)
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        sum_round = {"error": f"{type(e).__name__}: {e}"}
    # The serving stream and the deterministic baselines repeat one GPU's figures on every rank; with
    # several ranks (all GPUs held) they run only at N = 1.
    single_gpu = world == 1
    try:
        serving = (serving_run(B, args.serve_requests, args.streams, 120 << 30, args.serve_open_requests)
                   if (args.serve_requests > 0 or args.serve_open_requests > 0) and single_gpu else None)
    except Exception as e:  # noqa: BLE001
        serving = {"error": f"{type(e).__name__}: {e}"}

    # ---- deterministic FP64 TT-rounding on the same GPU (the comparison the metric names)
    det_ms, det_ranks, tdet_ms, tdet_ranks = [], None, [], None
    for i in range(args.det_steps + 1 if single_gpu else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with B.round_deterministic(cores, TOL) as z:
            det_ranks = z.ranks
        torch.cuda.synchronize()
        if i > 0:
            det_ms.append(1e3 * (time.perf_counter() - t0))

    # ---- the same algorithm on torch's FP64 cuSOLVER QR/SVD, as context for that comparison
    for i in range(max(1, args.det_steps) + 1 if single_gpu else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tdet_ranks = torch_deterministic(cores, TOL)
        torch.cuda.synchronize()
        if i > 0:
            tdet_ms.append(1e3 * (time.perf_counter() - t0))

    # ---- precision forms beside the headline's (slices from the tolerance, FP64 block loop): the
    # same single-stream rounding with the block loop in double-float, and at 8 slices
    # (FP64-accurate contractions)
    forms = {}
    what = {"sliced6_df_block_loop": "6 slices, the block loop's per-CTA arithmetic in double-float (FP32 pipe)",
            "sliced8_fp64": "8 slices (contractions FP64-accurate), FP64 block loop",
            "adap_r": "the headline form followed by the Remark 3.2 right-to-left compression pass (threshold tau), "
                      "which truncates the over-estimated ranks toward the deterministic rounding's"}
    if prec == B.TTR_PREC_SLICED:
        for name, kw in (("sliced6_df_block_loop", {"block_loop_df": True}), ("sliced8_fp64", {"slices": 8}),
                         ("adap_r", {"adap_r": True})):
            fo = B.options(precision=prec, nrmx=x.norm, **kw)
            for _ in range(2):
                B.round_adaptive(cores, TOL, BLOCK, SEED, fo).free()
            nf = max(3, min(args.steps, 30))
            fe = [torch.cuda.Event(enable_timing=True) for _ in range(nf + 1)]
            fe[0].record(stream)
            franks = None
            for i in range(nf):
                y = B.round_adaptive(cores, TOL, BLOCK, SEED, fo)
                franks = y.ranks
                y.free()
                fe[i + 1].record(stream)
            torch.cuda.synchronize()
            fms = [fe[i].elapsed_time(fe[i + 1]) for i in range(nf)]
            forms[name] = {"roundings_per_s": 1e3 * nf / fe[0].elapsed_time(fe[-1]),
                           "p50_ms": float(np.percentile(fms, 50)), "p99_ms": float(np.percentile(fms, 99)),
                           "steps": nf, "ranks_equal_headline": franks == out_ranks,
                           "max_rank": max(franks), "what": what[name],
                           "measured": "one rounding at a time on one stream (compare single_stream)"}

    # ---- end to end through host buffers: H2D of the cores, rounding, D2H of the result
    host = [torch.from_numpy(c).pin_memory() for c in x.cores]
    h2d = sum(c.nbytes for c in x.cores)
    # (a) one call at a time through tt_round_adaptive
    e2e_steps = max(3, min(args.steps, 10))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    d2h = 0
    for _ in range(e2e_steps):
        devc = [h.to("cuda", non_blocking=True) for h in host]
        with B.round_adaptive(devc, TOL, BLOCK, SEED, opts) as y:
            outs = [t.to("cpu") for t in y.to_torch()]
        d2h = sum(o.numel() * 8 for o in outs)
    torch.cuda.synchronize()
    e2e_single = e2e_steps / (time.perf_counter() - t0) * world
    # (b) through the request server, `streams` requests in flight: each request's H2D copy,
    # rounding and D2H copy overlap with the other requests' (the serving form of the metric)
    try:
        e2e_srv, d2h_srv, srv_steps = e2e_server_run(B, host, opts, args.streams, max(3, min(args.steps, 100)))
        e2e = {"value": e2e_srv * world, "unit": "roundings/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h_srv), "steps": srv_steps,
               "path": f"request server (ttr_server_*), {args.streams} workers; cores in pinned host memory"}
    except Exception as e:  # noqa: BLE001 - fall back to the one-call-at-a-time figure, and say so
        e2e = {"value": e2e_single, "unit": "roundings/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "path": "one call at a time (request server failed: "
               f"{type(e).__name__}: {e})"}

    line = {"metric": METRIC, "value": value, "unit": "roundings/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "latency": f"per rounding, host call to return, with {args.streams} roundings in flight",
            "single_stream": single, "sum_round": sum_round, "serving": serving,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else
            f"f64 via bf16 slices (tcgen05)", "data": "synthetic",
            "config": config(x, args.streams), "ranks_out": out_ranks, "sketch_width": w, "extensions": info["extensions"],
            "det_fp64": None if not det_ms else {
                "roundings_per_s": 1e3 / float(np.mean(det_ms)), "ms": float(np.mean(det_ms)), "ranks_out": det_ranks,
                "speedup_of_adaptive": value / world / (1e3 / float(np.mean(det_ms))),
                "note": "this library's Algorithm 1: Householder QR and multi-CTA one-sided Jacobi SVD, FP64"},
            "speedup_vs_fastest_deterministic": None if not (det_ms and tdet_ms) else
                value / world / (1e3 / min(float(np.mean(det_ms)), float(np.mean(tdet_ms)))),
            "precision_forms": forms or None,
            "det_torch_cusolver_fp64": None if not tdet_ms else {
                "ms": float(np.mean(tdet_ms)), "roundings_per_s": 1e3 / float(np.mean(tdet_ms)), "ranks_out": tdet_ranks,
                "note": "Algorithm 1 on torch.linalg.qr/svd (cuSOLVER), FP64, comparison only"},
            "roofline": roof, "roofline_other": roof_other[0] if roof_other else None, "gpu_launches": int(launches),
            "max_sms_per_stream": conc["max_sms_per_stream"], "measured_peaks_probe": probed,
            "e2e": e2e,
            "e2e_single_call": {"value": e2e_single, "unit": "roundings/s", "steps": e2e_steps,
                                "path": "tt_round_adaptive one call at a time: H2D, rounding, D2H in sequence"},
            "clocks": clk.summary()}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, n, dt = cpu_oracle_rate(x)
        line["cpu_baseline"] = {"value": v, "unit": "roundings/s", "cores": host_cores(), "kind": "oracle",
                                "sample": f"{n} whole adaptive roundings of the workload in {dt:.1f} s (numpy FP64)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
