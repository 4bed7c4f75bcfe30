#!/usr/bin/env python3
"""Benchmark of the OEM hot path on GB300.

Default workload (one "step" = the whole path over one synthetic problem):
n = 1,000,000 rows, p = 500, float32 X with AR(0.5) rows, 25 nonzero true
coefficients (|beta_j| ~ U[0.5, 2], random signs), noise sd 1; the X^T X /
X^T y pass (split-bfloat16 products on the tcgen05 tensor cores), d by
Lanczos, the lambda grids, and warm-started paths of 100 lambdas for four
penalties at once (lasso, elastic net alpha = 0.5, MCP gamma = 3, SCAD
gamma = 3.7), tol 1e-7. Metric: fitted paths per second.

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
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one ncu
# capture per kernel, for the bench workload's p = 500 at n = 200,000. The
# iteration reads its Gram once per launch (independent of n); the Gram pass
# moves bytes in proportion to n (scaled to the full n below). Set to None
# whenever the kernel changes, until it is captured again.
NCU_DRAM_BYTES = {"oem_iter_kernel": None,
                  "gram_tma_kernel_per_row": (419.602176e6 + 71.923456e6) / 200_000}

FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
WORKLOAD = "four_penalties_f32_n1e6_p500"


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

def oracle_step(w, n_sample: int, seed_shift: int = 0):
    """One bounded oracle step: the Gram of the first n_sample rows (its time
    scaled to the full n, the Gram being linear in n), d, lambda grids and
    the warm-started paths of every penalty on that Gram. Returns
    (scaled seconds, raw seconds)."""
    import oracle
    ww = synthgen.Workload(**{**w.__dict__, "seed": w.seed + seed_shift})
    X, y, _, _ = synthgen.make_data(ww, n=n_sample)
    t0 = time.perf_counter()
    G, c, N, n = oracle.gram_sums(synthgen.as_f64(X), y)
    t_gram = time.perf_counter() - t0
    G, c = G / n, c / n
    t1 = time.perf_counter()
    d = oracle.lanczos_d(G)[0]
    for kind, kw in penalties_of(w):
        pen = oracle.Penalty(kind, **kw)
        lams = oracle.lambda_grid(oracle.lambda_max(c, pen), w.nlambda, w.lambda_min_ratio)
        oracle.oem_path(G, c, d, pen, lams, tol=w.tol, max_iter=10000)
    t_rest = time.perf_counter() - t1
    return t_gram * (w.n / n_sample) + t_rest, t_gram + t_rest


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


def run_reference(args, w, rank, world):
    if rank != 0:
        return 0
    n_sample = min(w.n, args.cpu_sample_rows)
    npaths = len(w.penalties)
    for _ in range(args.warmup):
        oracle_step(w, n_sample)
    times = []
    for k in range(args.steps):
        s, _ = oracle_step(w, n_sample, seed_shift=0)
        times.append(s)
    total = sum(times)
    value = npaths * args.steps / total
    sample = (f"Gram of the first {n_sample} of {w.n} rows (time scaled by n/{n_sample}), then d "
              f"and {npaths} x {w.nlambda}-lambda paths on that Gram, per step")
    line = {
        "impl": "reference", "metric": "fitted paths/s", "value": value, "unit": "paths/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "p": w.p, "penalties": list(w.penalties),
                   "nlambda": w.nlambda, "tol": w.tol},
        "cpu_baseline": {"value": value, "unit": "paths/s", "cores": cpu_cores(), "cpu_model": cpu_model(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "paths/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

def run_ours(args, w, rank, world, local_rank):
    import torch
    import paper_1801_09661_gb300 as oem

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    ww = synthgen.Workload(**{**w.__dict__, "seed": w.seed + 1000 * rank})
    t0 = time.time()
    X, y, _, _ = synthgen.make_data(ww)
    t_gen = time.time() - t0
    Xd = oem.padded(X, device=dev)
    yd = torch.from_numpy(y).to(dev)
    pens = [oem.Penalty(k, **kw) for k, kw in penalties_of(w)]
    npen = len(pens)
    ctx = oem.Context(local_rank, budget_bytes=64 << 30)
    stream = torch.cuda.current_stream(dev)
    opts = dict(nlambda=w.nlambda, lambda_min_ratio=w.lambda_min_ratio, tol=w.tol,
                gram_mode=args.gram_mode)
    if args.cluster_ctas or args.instances_per_task:
        # a fixed iteration layout (no autotuning), e.g. for a profiler run,
        # where the autotuner's timing trials would be distorted
        opts.update(cluster_ctas=args.cluster_ctas, instances_per_task=args.instances_per_task,
                    autotune=False)
    beta, lam, its, conv = (torch.empty((npen, w.nlambda, w.p), dtype=torch.float64, device=dev),
                            torch.empty((npen, w.nlambda), dtype=torch.float64, device=dev),
                            torch.empty((npen, w.nlambda), dtype=torch.int32, device=dev),
                            torch.empty((npen, w.nlambda), dtype=torch.uint8, device=dev))
    dout = torch.empty(1, dtype=torch.float64, device=dev)
    out = (beta, lam, its, conv, dout)

    def step():
        oem.oem_fit(ctx, Xd, yd, pens, out=out, **opts)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    for _ in range(args.warmup):
        step()
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
    for _ in range(args.steps):
        step()
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
    its_h = its.cpu().numpy().astype(np.int64)
    conv_h = conv.cpu().numpy()
    loops = int(its_h.sum(axis=1).max())
    # ---------------- e2e: pinned host buffers, copies inside the timed region
    Xh = torch.from_numpy(np.ascontiguousarray(X)).pin_memory()
    yh = torch.from_numpy(y).pin_memory()
    bh = torch.empty(beta.shape, dtype=beta.dtype).pin_memory()
    lh = torch.empty(lam.shape, dtype=lam.dtype).pin_memory()
    ih = torch.empty(its.shape, dtype=its.dtype).pin_memory()
    ch = torch.empty(conv.shape, dtype=conv.dtype).pin_memory()
    # inputs double-buffered: the copy of step k + 1 (copy stream) overlaps
    # the fit of step k (compute stream); a buffer is refilled only after the
    # fit that read it; results are read back after each fit
    cs = torch.cuda.Stream(dev)
    xin = [(torch.empty_like(Xd), torch.empty_like(yd)) for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]
    for e in done:
        e.record(stream)

    def e2e_step(k):
        b = k % 2
        Xb, yb = xin[b]
        with torch.cuda.stream(cs):
            cs.wait_event(done[b])
            Xb.copy_(Xh, non_blocking=True)
            yb.copy_(yh, non_blocking=True)
            copied[b].record(cs)
        stream.wait_event(copied[b])
        oem.oem_fit(ctx, Xb, yb, pens, out=out, stream=stream.cuda_stream, **opts)
        bh.copy_(beta, non_blocking=True)
        lh.copy_(lam, non_blocking=True)
        ih.copy_(its, non_blocking=True)
        ch.copy_(conv, non_blocking=True)
        done[b].record(stream)

    e2e_step(0)
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    cs.wait_event(f0)
    for k in range(args.steps):
        e2e_step(k)
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms_e2e = f0.elapsed_time(f1)
    ms_e2e = max_over_ranks(ms_e2e, world, dev)
    h2d = Xh.numel() * Xh.element_size() + yh.numel() * yh.element_size()
    d2h = sum(t.numel() * t.element_size() for t in (bh, lh, ih, ch))

    # ---------------- X left in pinned host memory: the library streams it
    # through the Gram pass (row blocks copied while the previous block's pass
    # runs). Its bound is the host-to-device link, measured here by a plain
    # pinned copy of the same bytes.
    def timed(fn, reps):
        # median of single calls (one slow host-to-device transfer does not
        # move it)
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
            xin[0][0].copy_(Xh, non_blocking=True)

    def host_fit():
        oem.oem_fit(ctx, Xh, yh, pens, out=out, stream=stream.cuda_stream, **opts)
        with torch.cuda.stream(stream):
            bh.copy_(beta, non_blocking=True)
            lh.copy_(lam, non_blocking=True)

    streamed = None
    if Xh.stride(0) * Xh.element_size() % 16 == 0:  # the ABI's row-stride rule
        link_ms = timed(plain_copy, 5)
        sgram_ms = timed(lambda: oem.oem_gram(ctx, Xh, yh, stream=stream.cuda_stream), 5)
        hfit_ms = timed(host_fit, 5)
        link_gbs = X.nbytes / (link_ms / 1000.0) / 1e9
        sgram_gbs = X.nbytes / (sgram_ms / 1000.0) / 1e9
        streamed = {"entry": "oem_fit / oem_gram with X in pinned host memory (streamed Gram pass)",
                    "paths_per_s": npen / (hfit_ms / 1000.0), "ms_per_fit": hfit_ms,
                    "gram_ms": sgram_ms,
                    "roofline": {"bound": "h2d link", "achieved": sgram_gbs, "peak": link_gbs, "unit": "GB/s",
                                 "frac": sgram_gbs / link_gbs,
                                 "peak_source": "plain pinned copy of X timed in this run"}}

    if rank != 0:
        ctx.close()
        return 0
    peaks, peak_src = load_peaks()
    value = job_throughput(npen * args.steps, world, ms)
    # roofline: the OEM iteration kernel (dominant) against HBM
    p = w.p
    it_ms, it_n = prof.get("oem_iter_kernel", (float("nan"), 0))
    bytes_per_loop = p * (p + 1) / 2 * 4 + npen * 3 * p * 4
    it_bytes = loops * bytes_per_loop  # per launch (one launch per step)
    it_ms_launch = it_ms / max(1, it_n)
    it_gbs = it_bytes / (it_ms_launch / 1000.0) / 1e9
    hbm = float(peaks.get("hbm_gbs", FALLBACK_PEAKS["hbm_gbs"]))
    # the Gram pass (tensor cores): useful flops n (p+1)(p+2)
    gk = "gram_tc_pass" if "gram_tc_pass" in prof else "gram_simt_kernel"
    g_ms, g_n = prof.get(gk, (float("nan"), 0))
    # one pass per step (the TMA path is two launches: packing + SYRK)
    g_ms_launch = g_ms / max(1, args.steps)
    g_flops = w.n * (p + 1) * (p + 2)
    g_tf = g_flops / (g_ms_launch / 1000.0) / 1e12
    # MMA work: split mode takes four products on the nt diagonal tiles and
    # three on the nt (nt - 1) / 2 others; other modes one product per tile
    nt = math.ceil((p + 1) / 128)
    split = args.gram_mode in ("auto", "split_bf16")
    tile_products = (4 * nt + 3 * nt * (nt - 1) / 2) if split else nt * (nt + 1) / 2
    mma_flops = 2.0 * tile_products * 128 * 128 * w.n
    bf16 = float(peaks.get("bf16_tflops", FALLBACK_PEAKS["bf16_tflops"]))
    step_ms = ms / args.steps
    kernels = {k: {"ms_per_step": v[0] / args.steps, "launches_per_step": v[1] / args.steps,
                   "share": v[0] / max(1e-9, sum(x[0] for x in prof.values()))}
               for k, v in prof.items()}
    line = {
        "metric": "fitted paths/s", "value": value, "unit": "paths/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": w.name, "n": w.n, "p": p, "penalties": list(w.penalties),
                   "nlambda": w.nlambda, "lambda_min_ratio": w.lambda_min_ratio, "tol": w.tol,
                   "gram_mode": args.gram_mode, "x_dtype": w.dtype,
                   "iteration_layout": ({"cluster_ctas": args.cluster_ctas,
                                         "instances_per_task": args.instances_per_task}
                                        if args.cluster_ctas or args.instances_per_task else "autotuned"),
                   "l2": "inputs larger than L2 (X is %.2f GB)" % (X.nbytes / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": job_throughput(npen * args.steps, world, ms_e2e), "unit": "paths/s",
                "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "streamed": streamed,
        "roofline": {"kernel": "oem_iter_kernel", "bound": "hbm", "achieved": it_gbs, "peak": hbm,
                     "unit": "GB/s", "frac": it_gbs / hbm,
                     "traffic": NCU_DRAM_BYTES.get("oem_iter_kernel") if w.p == 500 else None,
                     "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": it_bytes, "loop_iterations": loops,
                     "ms_per_launch": it_ms_launch},
        "roofline_gram": {"kernel": gk, "bound": "tensor", "achieved": g_tf, "peak": bf16,
                          "unit": "TFLOP/s", "frac": g_tf / bf16,
                          "traffic": (NCU_DRAM_BYTES["gram_tma_kernel_per_row"] * w.n
                                      if w.p == 500 and NCU_DRAM_BYTES.get("gram_tma_kernel_per_row")
                                      and args.gram_mode in ("auto", "split_bf16") else None),
                          "peak_source": peak_src, "useful_flops": g_flops,
                          "mma_flops": mma_flops,
                          "mma_tflops": mma_flops / (g_ms_launch / 1000.0) / 1e12,
                          "ms_per_pass": g_ms_launch, "launches_per_pass": g_n / max(1, args.steps),
                          "hbm_gbs": X.nbytes / (g_ms_launch / 1000.0) / 1e9},
        "x_tx_tflops": g_tf,
        "kernels": kernels,
        "clocks": clk,
        "status": status,
        "converged_frac": float(conv_h.mean()),
        "datagen_s": t_gen,
    }
    # serving: Poisson arrivals of mixed fit / CV jobs, served (batched) vs plain
    if args.serving_requests > 0 and world == 1:
        served, same, sclk = serving_measure(args, rank, local_rank, args.serving_requests,
                                             args.plain_requests)
        line["serving"] = {"requests": served["requests"], "rate_per_s": args.rate,
                           "paths_per_s": served["paths_per_s"], "latency_ms": served["latency_ms"],
                           "batched_over_plain": same["batched_over_plain"],
                           "same_requests": same, "clocks": sclk}
    if not args.no_cpu_baseline:
        # the oracle on the full workload, repeated (fresh seeds) until about
        # 10 s of CPU work
        n_sample = min(w.n, args.cpu_sample_rows)
        tot_scaled, tot_raw, reps = 0.0, 0.0, 0
        while reps == 0 or tot_raw < args.cpu_seconds:
            scaled, raw = oracle_step(w, n_sample, seed_shift=reps)
            tot_scaled += scaled
            tot_raw += raw
            reps += 1
        line["cpu_baseline"] = {
            "value": npen * reps / tot_scaled, "unit": "paths/s", "cores": cpu_cores(), "cpu_model": cpu_model(), "kind": "oracle",
            "sample": (f"{reps} oracle steps, each the Gram of {n_sample} of {w.n} rows"
                       + (f" (time scaled by n/{n_sample})" if n_sample < w.n else "")
                       + f", d and {npen} x {w.nlambda}-lambda paths; {tot_raw:.1f} s of CPU work")}
    ctx.close()
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# Serving: Poisson arrivals of mixed fit / CV jobs, served (batched) vs plain
# ---------------------------------------------------------------------------

def serving_measure(args, rank, local_rank, nreq, nplain):
    """Requests arrive as a Poisson stream (50/s); each has n log-uniform in
    [1e4, 2e6], p uniform in [20, 1000], float32 AR(0.5) rows, 30% 5-fold CV,
    lasso or MCP (gamma 3) with 50 lambdas. The batched server admits them
    under a 150 GB budget and runs them with continuous batching; latency is
    submission -> results in host memory. The plain per-job form runs the
    first nplain of them (submitted at once) for the throughput comparison,
    against the batched form on the same requests. Returns (served,
    same_requests, clocks)."""
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
    lat = []
    for i in ids:
        st, l, rc = srv.wait(i, 3600)
        lat.append(l)
    wall = time.perf_counter() - t0
    clocks.mark(tw0, time.time())
    clk = clocks.stop()
    st_b = srv.stats()
    srv.close()
    total_paths = sum(paths_of(r) for r in reqs)
    lat = np.array(lat)
    served = {"paths_per_s": total_paths / wall, "wall_s": wall, "requests": len(reqs),
              "paths": total_paths, "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                                   "p99": float(np.percentile(lat, 99)),
                                                   "mean": float(lat.mean())},
              "rounds": st_b["rounds"], "kernel_launches": st_b["launches"],
              "peak_device_bytes": st_b["peak_bytes"]}

    # ---- throughput on the same requests: batched vs plain, all submitted at once
    m = min(nplain, len(reqs))
    out = {}
    for form in ("batched", "plain"):
        s2 = oem.Server(local_rank, budget_bytes=int(args.budget_gb * (1 << 30)), form=form,
                        iters_per_round=args.iters_per_round)
        t1 = time.perf_counter()
        ii = [submit(s2, reqs[k], data[k]) for k in range(m)]
        ll = [s2.wait(i, 7200)[1] for i in ii]
        w2 = time.perf_counter() - t1
        res = [s2.result(i) for i in ii]
        s2.close()
        out[form] = {"paths_per_s": sum(paths_of(reqs[k]) for k in range(m)) / w2, "wall_s": w2,
                     "p50_ms": float(np.percentile(ll, 50)), "p99_ms": float(np.percentile(ll, 99)),
                     "betas": [r["beta"] for r in res]}
    # equal accuracy: the two forms' paths agree (max |dbeta| relative to ||beta||_inf)
    acc = max(float(np.abs(a - b).max() / max(1.0, np.abs(b).max()))
              for a, b in zip(out["batched"]["betas"], out["plain"]["betas"]))
    for f in out.values():
        f.pop("betas")
    same = {"requests": m, "batched": out["batched"], "plain": out["plain"],
            "batched_over_plain": out["batched"]["paths_per_s"] / out["plain"]["paths_per_s"],
            "max_rel_beta_diff": acc}
    del bases, data
    torch.cuda.empty_cache()
    return served, same, clk


def run_serving(args, rank, world, local_rank):
    """The serving workload on its own line (see serving_measure)."""
    served, same, clk = serving_measure(args, rank, local_rank, args.requests, args.plain_requests)
    if rank != 0:
        return 0
    wall = served["wall_s"]
    nreq = served["requests"]
    line = {
        "metric": "fitted paths/s (served, Poisson arrivals)", "value": served["paths_per_s"],
        "unit": "paths/s", "n_gpus": world, "steps": nreq, "warmup": 0,
        "ms_per_step": 1000.0 * wall / nreq, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "serving", "requests": nreq, "rate_per_s": args.rate,
                   "n": "log-uniform [1e4, 2e6]", "p": "uniform [20, 1000]", "cv_frac": 0.3,
                   "K": 5, "nlambda": 50, "penalties": ["lasso", "mcp"],
                   "budget_gb": args.budget_gb, "iters_per_round": args.iters_per_round},
        "served": served,
        "same_requests": same,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(synthgen.WORKLOADS) + ["serving"])
    ap.add_argument("--requests", type=int, default=300, help="serving: number of requests")
    ap.add_argument("--rate", type=float, default=50.0, help="serving: arrivals per second")
    ap.add_argument("--plain-requests", type=int, default=40,
                    help="serving: requests in the batched-vs-plain comparison")
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--iters-per-round", type=int, default=1000)
    ap.add_argument("--cluster-ctas", type=int, default=0,
                    help="iteration layout: CTAs per task (0: autotuned)")
    ap.add_argument("--instances-per-task", type=int, default=0,
                    help="iteration layout: penalty paths per task (0: autotuned)")
    ap.add_argument("--gram-mode", default="auto",
                    choices=["auto", "split_bf16", "tf32", "fp32", "fp64", "bf16"])
    ap.add_argument("--cpu-sample-rows", type=int, default=1_000_000,
                    help="rows per oracle step of the CPU baseline (time scaled to n)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
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
