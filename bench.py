#!/usr/bin/env python3
"""Benchmark of the OEM hot path on GB300.

One "step" is the whole path over one synthetic problem: the X^T X / X^T y
pass (per fold for cross validation), d by Lanczos, the lambda grids and the
warm-started paths of every penalty (and every fold), all on the device.
Metric: fitted paths per second (a cross validation of K folds and m
penalties counts m (K + 1) paths).

Headline workload (the largest one that fits one GPU): group lasso on
n = 2,000,000 rows and p = 2,000 columns of bfloat16 X in 200 groups of 10
(correlation 0.7 inside a group, 0.2 across), 10 active groups, noise sd 2,
100 lambdas, tol 1e-7. The same JSON line carries, as sub-objects, the other
workloads measured the same way:
  * four penalties (lasso, elastic net 0.5, MCP 3, SCAD 3.7) on 10^6 x 500
    float32 AR(0.5) rows (split-bfloat16 Gram, 100 lambdas each);
  * 10-fold cross validation of the four penalties on 4 x 10^6 x 200 float32
    AR(0.5) rows (per-fold Grams in one pass, 44 paths);
  * the plain lasso on 10^4 x 50 float64 rows (latency-bound);
  * serving: 2,000 requests with Poisson arrivals (batched server against
    the plain per-job form and against sequential library calls).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 oracle (the plain CPU restatement of the
method) on the host cores on a bounded sample of the same workload.
Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthgen  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch from
# one ncu capture of each kernel, keyed by (kernel, workload): an iteration
# launch reads its Gram once (independent of n); Gram passes are given per
# row of X (bytes move in proportion to n). None until the current kernel has
# been captured.
NCU_DRAM_BYTES = {
    # profiles/oem_iter_rows_kernel_group_lasso_bf16_n2e5_p2000.md: 9.06 MB per
    # launch on the 2e5-row case (every touched 16-column block of G read
    # once); the iteration reads only the Gram, so a launch of the 2e6-row
    # workload moves the same
    ("oem_iter_rows_kernel", "group_lasso_bf16_n2e6_p2000"): 9.056512e6,
    ("oem_iter_rows_kernel", "group_lasso_bf16_n2e5_p2000"): 9.056512e6,
}

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
HEADLINE = "group_lasso_bf16_n2e6_p2000"
SECONDARY = ("four_penalties_f32_n1e6_p500", "cv10_f32_n4e6_p200", "lasso_f64_n1e4_p50")


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return d, "measured"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback"


def penalties_of(w):
    ex = w.extra
    out = []
    for k in w.penalties:
        if k == "enet":
            out.append(("enet", {"alpha": ex.get("alpha", 0.5)}))
        elif k == "mcp":
            out.append(("mcp", {"gamma": ex.get("gamma_mcp", 3.0)}))
        elif k == "scad":
            out.append(("scad", {"gamma": ex.get("gamma_scad", 3.7)}))
        elif k == "grp.lasso":
            out.append(("grp.lasso", {"groups": np.arange(w.p) // w.group_size}))
        else:
            out.append((k, {}))
    return out


def paths_per_step(w) -> int:
    return len(w.penalties) * ((w.K + 1) if w.K else 1)


class ClockSampler:
    """nvidia-smi samples (every 100 ms) with host timestamps. start() waits
    for the first sample so that the sampler is running when the timed region
    begins; mark(t0, t1) records the timed region; stop() keeps the samples
    inside it (or the nearest one when the region is shorter than the
    sampling period, flagged)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        import threading
        self.proc, self.lines, self.t0, self.t1 = None, [], None, None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        t_end = time.time() + 5.0
        while not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line))

    def mark(self, t0, t1):
        self.t0, self.t1 = t0, t1

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)  # one more period after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ts, line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((ts, float(f[1]), float(f[2]), f[5:9]))
            except ValueError:
                continue
        inside = [r for r in rows if self.t0 is not None and self.t0 <= r[0] <= self.t1 + 0.1]
        nearest = False
        if not inside and rows and self.t0 is not None:
            mid = 0.5 * (self.t0 + self.t1)
            inside = [min(rows, key=lambda r: abs(r[0] - mid))]
            nearest = True
        reasons = set()
        for r in inside:
            for nm, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        out = {"sm_mhz": statistics.median([r[1] for r in inside]) if inside else None,
               "sm_max_mhz": max(r[2] for r in inside) if inside else None,
               "samples": len(inside), "reasons": sorted(reasons)}
        if nearest:
            out["note"] = "timed region shorter than the 100 ms sampling period: nearest sample"
        return out


# ---------------------------------------------------------------------------
# FP64 oracle on the host (CPU baseline and the reference arm)
# ---------------------------------------------------------------------------

def _oracle_pens(w):
    import oracle
    return [oracle.Penalty(k, **kw) for k, kw in penalties_of(w)]


def oracle_gram_stats(w, n_sample: int, seed_shift: int = 0):
    """The oracle's Gram statistics of the first n_sample rows of the
    workload: (list of (G, c) scaled, seconds of the Gram sums). For cross
    validation the K fold sums, then the full and leave-fold-out Grams."""
    import oracle
    ww = synthgen.Workload(**{**w.__dict__, "seed": w.seed + seed_shift})
    X, y, fold, _ = synthgen.make_data(ww, n=n_sample)
    Xf = synthgen.as_f64(X)
    t0 = time.perf_counter()
    if w.K:
        Gk, ck, Nk, nk = oracle.fold_gram_sums(Xf, y, fold, w.K)
        t_gram = time.perf_counter() - t0
        G, c, _, _ = oracle.assemble_fold_grams(Gk, ck, Nk, nk)
        grams = [(G[b], c[b]) for b in range(w.K + 1)]
    else:
        G, c, _, n = oracle.gram_sums(Xf, y)
        t_gram = time.perf_counter() - t0
        grams = [(G / n, c / n)]
    return grams, t_gram


def oracle_path_sample(grams, w, max_iters: int):
    """Run the oracle's warm-started paths (every Gram, every penalty, the
    full-data lambda grid) until max_iters OEM iterations in total have run
    (max_iters <= 0: to the end). Returns (seconds of Lanczos, seconds of the
    iterations, iterations run, whether every path finished)."""
    import oracle
    pens = _oracle_pens(w)
    t0 = time.perf_counter()
    ds = [oracle.lanczos_d(G)[0] for G, _ in grams]
    t_lz = time.perf_counter() - t0
    c0 = grams[0][1]
    lams = [oracle.lambda_grid(oracle.lambda_max(c0, pen), w.nlambda, w.lambda_min_ratio) for pen in pens]
    t1 = time.perf_counter()
    done, total = True, 0
    for (G, c), d in zip(grams, ds):
        for pen, lam in zip(pens, lams):
            beta = None
            for l in range(w.nlambda):
                left = max_iters - total if max_iters > 0 else 10_000
                if left <= 0:
                    done = False
                    break
                r = oracle.oem_path(G, c, d, pen, lam[l:l + 1], tol=w.tol,
                                    max_iter=min(10_000, left), beta0=beta)
                beta = r.beta[0]
                total += int(r.iters[0])
            if not done:
                break
        if not done:
            break
    return t_lz, time.perf_counter() - t1, total, done


def oracle_step(w, n_sample: int, total_iters: int, iter_sample: int, seed_shift: int = 0):
    """One bounded oracle step of workload w: the Gram of n_sample rows (time
    scaled by n / n_sample, the Gram being linear in n), d of every Gram, and
    iter_sample OEM iterations of the paths (time scaled by total_iters /
    iter_sample, the iterations of one path costing alike). Returns
    (scaled seconds of one whole step, raw seconds)."""
    grams, t_gram = oracle_gram_stats(w, n_sample, seed_shift)
    t_lz, t_it, its, done = oracle_path_sample(grams, w, iter_sample)
    t_path = t_it if done else t_it * total_iters / max(1, its)
    return t_gram * (w.n / n_sample) + t_lz + t_path, t_gram + t_lz + t_it


def oracle_total_iters(w, n_sample: int) -> int:
    """OEM iterations of the whole step as the oracle runs it (every path to
    the end on the Gram of n_sample rows)."""
    grams, _ = oracle_gram_stats(w, n_sample)
    return oracle_path_sample(grams, w, 0)[2]


def max_over_ranks(ms: float, world: int, device="cpu") -> float:
    """The slowest rank's time for the timed region (every rank leaves it at
    the same barrier; the job is as fast as its last rank)."""
    if world <= 1:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_throughput(paths_per_rank: int, world: int, ms: float) -> float:
    """Whole-job paths/s: the paths of every rank over the slowest rank's time."""
    return paths_per_rank * world / (ms / 1000.0)


def cpu_cores():
    return os.cpu_count() or 1


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.machine()


def cpu_baseline(w, total_iters: int, args, source: str):
    """The oracle on a bounded sample of workload w, repeated (fresh seeds)
    until args.cpu_seconds of CPU work; paths/s of whole steps."""
    n_sample = min(w.n, args.cpu_sample_rows)
    tot_scaled, tot_raw, reps = 0.0, 0.0, 0
    while reps == 0 or tot_raw < args.cpu_seconds:
        scaled, raw = oracle_step(w, n_sample, total_iters, args.cpu_iters, seed_shift=reps)
        tot_scaled += scaled
        tot_raw += raw
        reps += 1
    npaths = paths_per_step(w)
    sample = (f"{reps} oracle steps, each the Gram of {n_sample} of {w.n} rows"
              + (f" (time scaled by n/{n_sample})" if n_sample < w.n else "")
              + f", d of every Gram and up to {args.cpu_iters} OEM iterations of the {npaths} paths"
              + f" (time scaled to the {total_iters} iterations of a whole step, {source});"
              + f" {tot_raw:.1f} s of CPU work")
    return {"value": npaths * reps / tot_scaled, "unit": "paths/s", "cores": cpu_cores(),
            "cpu_model": cpu_model(), "kind": "oracle", "sample": sample}


# OEM iterations of a whole step as the oracle runs it (every path to its end
# on the Gram of the first 200,000 rows), counted once by oracle_total_iters:
# the count takes minutes at p = 2,000 (every iteration a dense 2,000 x 2,000
# mat-vec), so the reference arm uses the stored count for that workload.
ORACLE_TOTAL_ITERS = {"group_lasso_bf16_n2e6_p2000": 426460}


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    n_sample = min(w.n, args.cpu_sample_rows)
    it_sample = args.cpu_iters
    npaths = paths_per_step(w)
    # the iterations of a whole step, counted by the oracle itself (untimed)
    total = ORACLE_TOTAL_ITERS.get(w.name) or oracle_total_iters(w, n_sample)
    # every step is a bounded sample: after the first warm-up step the
    # sample shrinks (rows of the Gram, OEM iterations) so that one step
    # takes about `target` seconds and the whole run a few minutes
    target = max(3.0, 150.0 / max(1, args.steps + args.warmup))
    for k in range(args.warmup):
        _, raw = oracle_step(w, n_sample, total, it_sample)
        if k == 0 and raw > target:
            f = target / raw
            n_sample = max(min(w.n, 5000), int(n_sample * f))
            it_sample = max(200, int(it_sample * f))
    times = []
    for _ in range(args.steps):
        s, _ = oracle_step(w, n_sample, total, it_sample)
        times.append(s)
    tot = sum(times)
    value = npaths * args.steps / tot
    sample = (f"per step the Gram of the first {n_sample} of {w.n} rows (time scaled by n/{n_sample}), "
              f"d of every Gram and up to {it_sample} OEM iterations of the {npaths} paths "
              f"(time scaled to the {total} iterations of a whole step, counted by the oracle)")
    line = {
        "impl": "reference", "metric": "fitted paths/s", "value": value, "unit": "paths/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w),
        "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cpu_cores(), "cpu_model": cpu_model(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def workload_config(w):
    cfg = {"workload": w.name, "n": w.n, "p": w.p, "x_dtype": w.dtype,
           "penalties": list(w.penalties), "nlambda": w.nlambda,
           "lambda_min_ratio": w.lambda_min_ratio, "tol": w.tol}
    if w.K:
        cfg["folds"] = w.K
    if w.group_size:
        cfg["group_size"] = w.group_size
    return cfg


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def to_device(oem, X, dev):
    """X on the device with a 16-byte row stride (bfloat16 bits as bfloat16)."""
    import torch
    if X.dtype == np.uint16:
        return oem.padded(torch.from_numpy(X.view(np.int16)).view(torch.bfloat16), device=dev)
    return oem.padded(X, device=dev)


def to_pinned(X):
    import torch
    if X.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(X).view(np.int16)).view(torch.bfloat16).pin_memory()
    return torch.from_numpy(np.ascontiguousarray(X)).pin_memory()


def iteration_bytes(w) -> float:
    """Algorithmic bytes of one OEM iteration of every instance of a step:
    the float32 upper triangle of each Gram, and c, beta in, beta out of each
    instance (float32)."""
    B = (w.K + 1) if w.K else 1
    p = w.p
    return B * (p * (p + 1) / 2 * 4 + len(w.penalties) * 3 * p * 4)


def measure_workload(args, w, rank, world, local_rank, steps, warmup, gram_mode="auto",
                     with_e2e=True, with_streamed=False, with_cpu=True):
    """Time `steps` whole-path steps of workload w on the device (inputs
    resident), then end to end from pinned host memory; per-kernel times from
    the library's event profiler; rooflines of the iteration and the Gram
    pass. Returns the result dict (rank 0) or None."""
    import torch
    import paper_1801_09661_gb300 as oem

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ww = synthgen.Workload(**{**w.__dict__, "seed": w.seed + 1000 * rank})
    t0 = time.time()
    X, y, fold, _ = synthgen.make_data(ww)
    t_gen = time.time() - t0
    Xd = to_device(oem, X, dev)
    yd = torch.from_numpy(y).to(dev)
    fd = torch.from_numpy(fold).to(dev) if w.K else None
    pens = [oem.Penalty(k, **kw) for k, kw in penalties_of(w)]
    npen = len(pens)
    L = w.nlambda
    ctx = oem.Context(local_rank, budget_bytes=64 << 30)
    stream = torch.cuda.current_stream(dev)
    opts = dict(nlambda=L, lambda_min_ratio=w.lambda_min_ratio, tol=w.tol, gram_mode=gram_mode)
    if args.cluster_ctas or args.instances_per_task:
        # a fixed iteration layout (no autotuning), e.g. for a profiler run,
        # where the autotuner's timing trials would be distorted
        opts.update(cluster_ctas=args.cluster_ctas, instances_per_task=args.instances_per_task,
                    autotune=False)
    if w.K:
        out = oem.cv_outputs(npen, L, w.p, dev)

        def fit(Xa, ya, fa, s=None):
            oem.oem_cv(ctx, Xa, ya, fa, w.K, pens, out=out, stream=s, **opts)
        its_t, conv_t = None, None
        res = [out[k] for k in ("beta", "lambdas", "cvm", "cvsd", "idx_min", "idx_1se", "best_penalty")]
    else:
        beta = torch.empty((npen, L, w.p), dtype=torch.float64, device=dev)
        lam = torch.empty((npen, L), dtype=torch.float64, device=dev)
        its_t = torch.empty((npen, L), dtype=torch.int32, device=dev)
        conv_t = torch.empty((npen, L), dtype=torch.uint8, device=dev)
        dout = torch.empty(1, dtype=torch.float64, device=dev)
        fout = (beta, lam, its_t, conv_t, dout)

        def fit(Xa, ya, fa, s=None):
            oem.oem_fit(ctx, Xa, ya, pens, out=fout, stream=s, **opts)
        res = [beta, lam, its_t, conv_t]

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(warmup):
        fit(Xd, yd, fd)
    ctx.sync()
    # ---------------- timed region: device-resident inputs
    clocks = ClockSampler(local_rank)
    ctx.profile(True)
    l0 = ctx.launches()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    e0.record(stream)
    for _ in range(steps):
        fit(Xd, yd, fd)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark(tw0, time.time())
    barrier()
    ms = e0.elapsed_time(e1)
    launches = ctx.launches() - l0
    prof = ctx.profile_read()
    ctx.profile(False)
    clk = clocks.stop()
    status = ctx.sync()
    ms = max_over_ranks(ms, world, dev)
    # OEM iterations of the last step (every instance) and the loop trips of
    # its iteration launch
    iters_total, loops = ctx.iter_stats()
    conv_frac = float(conv_t.float().mean().item()) if conv_t is not None else None

    e2e = None
    if with_e2e:
        # pinned host buffers, copies inside the timed region; inputs
        # double-buffered: the copy of step k + 1 (copy stream) overlaps the
        # fit of step k (compute stream); a buffer is refilled only after the
        # fit that read it; results are read back after each fit
        Xh, yh = to_pinned(X), torch.from_numpy(y).pin_memory()
        fh = torch.from_numpy(fold).pin_memory() if w.K else None
        rh = [torch.empty(t.shape, dtype=t.dtype).pin_memory() for t in res]
        cs = torch.cuda.Stream(dev)
        xin = [(torch.empty_like(Xd), torch.empty_like(yd), torch.empty_like(fd) if w.K else None)
               for _ in range(2)]
        copied = [torch.cuda.Event() for _ in range(2)]
        done = [torch.cuda.Event() for _ in range(2)]
        for e in done:
            e.record(stream)

        def e2e_step(k):
            b = k % 2
            Xb, yb, fb = xin[b]
            with torch.cuda.stream(cs):
                cs.wait_event(done[b])
                Xb.copy_(Xh, non_blocking=True)
                yb.copy_(yh, non_blocking=True)
                if w.K:
                    fb.copy_(fh, non_blocking=True)
                copied[b].record(cs)
            stream.wait_event(copied[b])
            fit(Xb, yb, fb, stream.cuda_stream)
            with torch.cuda.stream(stream):
                for h, t in zip(rh, res):
                    h.copy_(t, non_blocking=True)
            done[b].record(stream)

        e2e_step(0)
        torch.cuda.synchronize()
        barrier()
        torch.cuda.synchronize()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        cs.wait_event(f0)
        for k in range(steps):
            e2e_step(k)
        f1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ms_e2e = max_over_ranks(f0.elapsed_time(f1), world, dev)
        h2d = Xh.numel() * Xh.element_size() + yh.numel() * yh.element_size()
        if w.K:
            h2d += fh.numel() * fh.element_size()
        d2h = sum(t.numel() * t.element_size() for t in rh)
        e2e = {"value": job_throughput(paths_per_step(w) * steps, world, ms_e2e), "unit": "paths/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}
        del xin, Xh

    streamed = None
    if with_streamed and not w.K:
        streamed = measure_streamed(oem, ctx, X, y, pens, opts, fout, stream)

    if rank != 0:
        ctx.close()
        return None
    peaks, peak_src = load_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    bf16 = float(peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]))
    p = w.p
    step_ms = ms / steps
    # ---- the OEM iteration against HBM (its algorithmic bytes per loop trip)
    it_ms, it_n = prof.get("oem_iter_kernel", (float("nan"), 0))
    it_ms_step = it_ms / steps
    it_bytes = loops * iteration_bytes(w)
    it_gbs = it_bytes / (it_ms_step / 1000.0) / 1e9
    # the replicated-update kernel serves p <= 1024, the row-owned one beyond
    it_kernel = "oem_iter_kernel" if p <= 1024 else "oem_iter_rows_kernel"
    roofline = {"kernel": it_kernel, "bound": "hbm", "achieved": it_gbs, "peak": hbm,
                "unit": "GB/s", "frac": it_gbs / hbm,
                "traffic": NCU_DRAM_BYTES.get((it_kernel, w.name)),
                "peak_source": peak_src, "algorithmic_bytes_per_step": it_bytes,
                "algorithmic_bytes_per_loop": iteration_bytes(w), "loop_iterations": loops,
                "oem_iterations": iters_total, "ms_per_step": it_ms_step,
                "launches_per_step": it_n / steps,
                "us_per_loop": 1000.0 * it_ms_step / max(1, loops)}
    # ---- the Gram pass: useful flops n (p+1)(p+2) (upper triangle of [X|y]);
    # tensor-bound against the bf16 peak, except where its intensity is below
    # the ridge (the 4e6 x 200 cross validation: HBM-bound)
    gk = "gram_tc_pass" if "gram_tc_pass" in prof else "gram_simt_kernel"
    g_ms, g_n = prof.get(gk, (float("nan"), 0))
    g_ms_pass = g_ms / steps
    g_flops = w.n * (p + 1) * (p + 2)
    g_tf = g_flops / (g_ms_pass / 1000.0) / 1e12
    elem = {"f64": 8, "f32": 4, "bf16": 2}[w.dtype]
    g_bytes = w.n * p * elem + y.nbytes + (fold.nbytes if w.K else 0)
    g_gbs = g_bytes / (g_ms_pass / 1000.0) / 1e9
    intensity = g_flops / g_bytes
    hbm_bound = intensity < bf16 * 1e12 / (hbm * 1e9) / (3.0 if w.dtype == "f32" else 1.0)
    if hbm_bound:
        roofline_gram = {"kernel": gk, "bound": "hbm", "achieved": g_gbs, "peak": hbm, "unit": "GB/s",
                         "frac": g_gbs / hbm, "tflops": g_tf}
    else:
        roofline_gram = {"kernel": gk, "bound": "tensor", "achieved": g_tf, "peak": bf16,
                         "unit": "TFLOP/s", "frac": g_tf / bf16, "hbm_gbs": g_gbs}
    roofline_gram.update({"traffic": NCU_DRAM_BYTES.get((gk, w.name)), "peak_source": peak_src,
                          "useful_flops": g_flops, "algorithmic_bytes": g_bytes,
                          "ms_per_pass": g_ms_pass, "launches_per_pass": g_n / steps})
    tot_prof = sum(x[0] for x in prof.values())
    kernels = {k: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps,
                   "share": v[0] / max(1e-9, tot_prof)} for k, v in prof.items()}
    out = {
        "workload": w.name, "value": job_throughput(paths_per_step(w) * steps, world, ms),
        "unit": "paths/s", "ms_per_step": step_ms, "steps": steps, "warmup": warmup,
        "config": {**workload_config(w), "gram_mode": gram_mode,
                   "iteration_layout": ({"cluster_ctas": args.cluster_ctas,
                                         "instances_per_task": args.instances_per_task}
                                        if args.cluster_ctas or args.instances_per_task else "autotuned"),
                   "l2": "inputs larger than L2 (X is %.2f GB)" % (X.nbytes / 1e9)
                   if X.nbytes > 129e6 else "X (%.1f MB) fits in L2; L2 not flushed" % (X.nbytes / 1e6)},
        "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "roofline_gram": roofline_gram,
        "x_tx_tflops": g_tf, "kernels": kernels, "clocks": clk, "status": status,
        "converged_frac": conv_frac, "datagen_s": t_gen,
    }
    if streamed is not None:
        out["streamed"] = streamed
    ctx.close()
    if with_cpu and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, iters_total, args,
                                           "the iteration count of this run's last step")
    return out


def measure_streamed(oem, ctx, X, y, pens, opts, fout, stream):
    """X left in pinned host memory: the library streams it through the Gram
    pass (row blocks copied while the previous block's pass runs). Its bound
    is the host-to-device link, measured here by a plain pinned copy of the
    same bytes."""
    import torch
    Xh = to_pinned(X)
    yh = torch.from_numpy(y).pin_memory()
    if Xh.stride(0) * Xh.element_size() % 16:
        return None
    buf = torch.empty(Xh.shape, dtype=Xh.dtype, device=fout[0].device)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def plain_copy():
        with torch.cuda.stream(stream):
            buf.copy_(Xh, non_blocking=True)

    def host_fit():
        oem.oem_fit(ctx, Xh, yh, pens, out=fout, stream=stream.cuda_stream, **opts)

    link_ms = timed(plain_copy, 5)
    sgram_ms = timed(lambda: oem.oem_gram(ctx, Xh, yh, stream=stream.cuda_stream), 5)
    hfit_ms = timed(host_fit, 5)
    link_gbs = X.nbytes / (link_ms / 1000.0) / 1e9
    sgram_gbs = X.nbytes / (sgram_ms / 1000.0) / 1e9
    return {"entry": "oem_fit / oem_gram with X in pinned host memory (streamed Gram pass)",
            "paths_per_s": len(pens) / (hfit_ms / 1000.0), "ms_per_fit": hfit_ms, "gram_ms": sgram_ms,
            "roofline": {"bound": "h2d link", "achieved": sgram_gbs, "peak": link_gbs, "unit": "GB/s",
                         "frac": sgram_gbs / link_gbs,
                         "peak_source": "plain pinned copy of X timed in this run"}}


def run_ours(args, w, rank, world, local_rank):
    main = measure_workload(args, w, rank, world, local_rank, args.steps, args.warmup,
                            gram_mode=args.gram_mode, with_streamed=(w.name == "four_penalties_f32_n1e6_p500"))
    subs = {}
    if not args.headline_only:
        for name in SECONDARY:
            if name == w.name:
                continue
            sw = synthgen.WORKLOADS[name]
            subs[name] = measure_workload(args, sw, rank, world, local_rank, args.steps, args.warmup,
                                          with_streamed=(name == "four_penalties_f32_n1e6_p500"))
    serving = None
    if args.serving_requests > 0 and world == 1:
        serving = serving_measure(args, rank, local_rank, args.serving_requests, args.plain_requests)
    if rank != 0:
        return 0
    line = {
        "metric": "fitted paths/s", "value": main["value"], "unit": "paths/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (bf16 X, f32 iteration)" if w.dtype == "bf16" else "f32", "data": "synthetic",
        "config": {**main["config"], "parallelism": "replicas" if world > 1 else "single"},
        "e2e": main["e2e"], "gpu_launches": main["gpu_launches"],
        "roofline": main["roofline"], "roofline_gram": main["roofline_gram"],
        "x_tx_tflops": main["x_tx_tflops"], "kernels": main["kernels"], "clocks": main["clocks"],
        "status": main["status"], "converged_frac": main["converged_frac"], "datagen_s": main["datagen_s"],
    }
    if "cpu_baseline" in main:
        line["cpu_baseline"] = main["cpu_baseline"]
    if "streamed" in main:
        line["streamed"] = main["streamed"]
    if subs:
        line["workloads"] = subs
    if serving is not None:
        line["serving"] = serving
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Serving: Poisson arrivals of mixed fit / CV jobs
# ---------------------------------------------------------------------------

def serving_measure(args, rank, local_rank, nreq, nplain):
    """Requests arrive as a Poisson stream (50/s); each has n log-uniform in
    [1e4, 2e6], p uniform in [20, 1000], float32 AR(0.5) rows, 30% 5-fold CV,
    lasso or MCP (gamma 3) with 50 lambdas. The batched server admits them
    under a 150 GB budget and runs them with continuous batching; latency is
    submission -> results in host memory.
      * served: the Poisson stream through the batched server;
      * saturated: the first nsat requests submitted at once (the server's
        capacity and its latency when it is never idle);
      * same_requests: the first nplain requests submitted at once through
        the batched server, the plain per-job form (one launch per OEM
        iteration, float32 CUDA-core Gram), and one at a time through the
        library's own fit / cross-validation calls (oem_fit, oem_cv: split
        bfloat16 Gram, one persistent iteration launch per job; no batching
        across jobs)."""
    import torch
    import paper_1801_09661_gb300 as oem
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    reqs = synthgen.serving_requests(nreq, seed=5 + 1000 * rank, rate_per_s=args.rate)
    n_max = max(r["n"] for r in reqs)
    bases = [synthgen.device_ar1_base(n_max, 1000, 0.5, 77 + b, device=dev) for b in range(2)]
    data = [synthgen.device_request_data(bases[r["id"] % 2], r) for r in reqs]
    torch.cuda.synchronize()

    def submit(srv, r, d):
        X, y, fold = d
        pen = oem.Penalty(r["penalty"], gamma=r["gamma"])
        return srv.submit(X, y, pen, fold=fold, K=r["K"], nlambda=r["nlambda"], tol=1e-7,
                          gram_mode="auto")

    def paths_of(r):
        return r["K"] + 1 if r["K"] else 1

    def lat_stats(lat):
        lat = np.asarray(lat)
        return {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                "mean": float(lat.mean())}

    # ---- served, Poisson arrivals
    srv = oem.Server(local_rank, budget_bytes=int(args.budget_gb * (1 << 30)), form="batched",
                     iters_per_round=args.iters_per_round)
    clocks = ClockSampler(local_rank)
    tw0 = time.time()
    t0 = time.perf_counter()
    ids = []
    for r, d in zip(reqs, data):
        dt = r["arrival_s"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        ids.append(submit(srv, r, d))
    lat = [srv.wait(i, 3600)[1] for i in ids]
    wall = time.perf_counter() - t0
    clocks.mark(tw0, time.time())
    clk = clocks.stop()
    st_b = srv.stats()
    srv.close()
    total_paths = sum(paths_of(r) for r in reqs)
    served = {"paths_per_s": total_paths / wall, "wall_s": wall, "requests": len(reqs),
              "paths": total_paths, "latency_ms": lat_stats(lat),
              "rounds": st_b["rounds"], "kernel_launches": st_b["launches"],
              "peak_device_bytes": st_b["peak_bytes"]}

    # ---- saturated: all at once
    nsat = min(args.saturated_requests, len(reqs))
    saturated = None
    if nsat > 0:
        s3 = oem.Server(local_rank, budget_bytes=int(args.budget_gb * (1 << 30)), form="batched",
                        iters_per_round=args.iters_per_round)
        t1 = time.perf_counter()
        ii = [submit(s3, reqs[k], data[k]) for k in range(nsat)]
        ll = [s3.wait(i, 7200)[1] for i in ii]
        w3 = time.perf_counter() - t1
        s3.close()
        saturated = {"requests": nsat, "paths_per_s": sum(paths_of(reqs[k]) for k in range(nsat)) / w3,
                     "wall_s": w3, "latency_ms": lat_stats(ll),
                     "note": "every request submitted at time 0: latency includes the wait for admission"}

    # ---- the same requests through the three forms
    m = min(nplain, len(reqs))
    forms = {}
    betas = {}
    for form in ("batched", "plain"):
        s2 = oem.Server(local_rank, budget_bytes=int(args.budget_gb * (1 << 30)), form=form,
                        iters_per_round=args.iters_per_round)
        t1 = time.perf_counter()
        ii = [submit(s2, reqs[k], data[k]) for k in range(m)]
        ll = [s2.wait(i, 7200)[1] for i in ii]
        w2 = time.perf_counter() - t1
        betas[form] = [s2.result(i)["beta"] for i in ii]
        s2.close()
        forms[form] = {"paths_per_s": sum(paths_of(reqs[k]) for k in range(m)) / w2, "wall_s": w2,
                       "p50_ms": float(np.percentile(ll, 50)), "p99_ms": float(np.percentile(ll, 99))}
    # one job at a time through oem_fit / oem_cv (each job's layout by the
    # default rule: every job has a new shape, so nothing is autotuned)
    ctx = oem.Context(local_rank, budget_bytes=int(args.budget_gb * (1 << 30)))
    seq_b, ll = [], []
    t1 = time.perf_counter()
    for k in range(m):
        r = reqs[k]
        X, y, fold = data[k]
        pen = [oem.Penalty(r["penalty"], gamma=r["gamma"])]
        kw = dict(nlambda=r["nlambda"], tol=1e-7, gram_mode="auto", autotune=False)
        if r["K"]:
            o = oem.oem_cv(ctx, X, y, fold, r["K"], pen, **kw)
            b = o["beta"]
        else:
            b = oem.oem_fit(ctx, X, y, pen, **kw)[0]
        ctx.sync()
        seq_b.append(b[0].cpu().numpy())
        ll.append(1000.0 * (time.perf_counter() - t1))
    w2 = time.perf_counter() - t1
    ctx.close()
    forms["sequential_fit"] = {"paths_per_s": sum(paths_of(reqs[k]) for k in range(m)) / w2, "wall_s": w2,
                               "p50_ms": float(np.percentile(ll, 50)), "p99_ms": float(np.percentile(ll, 99)),
                               "entry": "oem_fit / oem_cv, one job at a time, results read back per job"}

    # equal accuracy: the forms' full-data paths agree (max |dbeta| relative to ||beta||_inf)
    def rel(a, b):
        a = np.asarray(a).reshape(-1, np.asarray(a).shape[-1])
        b = np.asarray(b).reshape(-1, np.asarray(b).shape[-1])
        a = a[: b.shape[0]]
        return float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))
    acc_plain = max(rel(a, b) for a, b in zip(betas["batched"], betas["plain"]))
    acc_seq = max(rel(np.asarray(a).reshape(-1, a.shape[-1])[: b.shape[0]], b)
                  for a, b in zip(betas["batched"], seq_b))
    same = {"requests": m, **forms,
            "batched_over_plain": forms["batched"]["paths_per_s"] / forms["plain"]["paths_per_s"],
            "batched_over_sequential_fit": forms["batched"]["paths_per_s"] / forms["sequential_fit"]["paths_per_s"],
            "max_rel_beta_diff_plain": acc_plain, "max_rel_beta_diff_sequential": acc_seq}
    del bases, data
    torch.cuda.empty_cache()
    return {"requests": served["requests"], "rate_per_s": args.rate,
            "paths_per_s": served["paths_per_s"], "latency_ms": served["latency_ms"],
            "served": served, "saturated": saturated, "same_requests": same,
            "batched_over_plain": same["batched_over_plain"],
            "batched_over_sequential_fit": same["batched_over_sequential_fit"], "clocks": clk}


def run_serving(args, rank, world, local_rank):
    """The serving workload on its own line (see serving_measure)."""
    s = serving_measure(args, rank, local_rank, args.requests, args.plain_requests)
    if rank != 0:
        return 0
    served = s["served"]
    nreq = served["requests"]
    line = {
        "metric": "fitted paths/s (served, Poisson arrivals)", "value": served["paths_per_s"],
        "unit": "paths/s", "n_gpus": world, "steps": nreq, "warmup": 0,
        "ms_per_step": 1000.0 * served["wall_s"] / nreq, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving", "requests": nreq, "rate_per_s": args.rate,
                   "n": "log-uniform [1e4, 2e6]", "p": "uniform [20, 1000]", "cv_frac": 0.3,
                   "K": 5, "nlambda": 50, "penalties": ["lasso", "mcp"],
                   "budget_gb": args.budget_gb, "iters_per_round": args.iters_per_round},
        **{k: v for k, v in s.items() if k not in ("requests", "rate_per_s", "paths_per_s")},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=HEADLINE, choices=sorted(synthgen.WORKLOADS) + ["serving"])
    ap.add_argument("--headline-only", action="store_true",
                    help="measure only --workload (no secondary workloads)")
    ap.add_argument("--requests", type=int, default=300, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=50.0, help="serving: arrivals per second")
    ap.add_argument("--plain-requests", type=int, default=40,
                    help="serving: requests in the batched / plain / sequential comparison")
    ap.add_argument("--saturated-requests", type=int, default=400,
                    help="serving: requests submitted at once for the saturation run")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--iters-per-round", type=int, default=1000)
    ap.add_argument("--cluster-ctas", type=int, default=0,
                    help="iteration layout: CTAs per task (0: autotuned)")
    ap.add_argument("--instances-per-task", type=int, default=0,
                    help="iteration layout: penalty paths per task (0: autotuned)")
    ap.add_argument("--gram-mode", default="auto",
                    choices=["auto", "split_bf16", "tf32", "fp32", "fp64", "bf16"])
    ap.add_argument("--cpu-sample-rows", type=int, default=200_000,
                    help="rows of the Gram in each oracle step (time scaled to n)")
    ap.add_argument("--cpu-iters", type=int, default=20_000,
                    help="OEM iterations run in each oracle step (time scaled to the whole step)")
    ap.add_argument("--cpu-seconds", type=float, default=8.0,
                    help="CPU baseline: repeat oracle steps until this much CPU work")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests of the serving measurement added to the default line (0: none)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.workload == "serving":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable":
                              "serving is a GPU request loop; the oracle has no serving form "
                              "(run the default workload for the oracle reference arm)"}))
            return 0
        return run_serving(args, rank, world, local_rank)
    w = synthgen.WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, w, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    rc = run_ours(args, w, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
