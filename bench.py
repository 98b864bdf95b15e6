"""Benchmark of the fused generate-and-sketch hot path.

One step = the left sketches Y = S A of the tall-skinny workload
(A 2^20 x 512 FP32 ~ N(0,1), k = 2048) with a Rademacher and with a
Gaussian S, both regenerated inside the kernels from Philox4x32-10.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--form bf16x2|fp32|fp8]
                  [--impl ours|reference] [--workload C1|C2|C3|C4|C5|NYS]

C1-C3 time single sketches, C4 a batch of 256 sketches in one persistent
launch, C5 the request server under a Poisson stream (latency percentiles),
NYS the Nystrom pair (B = A Omega, C = Omega^T B) of a 50000 x 50000 RBF
kernel matrix.

Prints ONE JSON line (rank 0).  `value` is useful TFLOP/s (2 k m n per
sketch) over the whole job; `roofline` describes the dominant kernel (the
fused sketch kernel) timed with CUDA events recorded by the library's
measurement hook around each of its launches; `e2e` repeats the step
through the host-buffer entry points (A copied host->device and Y copied
back inside the timed region); `cpu_baseline` is the CPU oracle on a
bounded sample of whole rows.  `--impl reference` times the CPU oracle alone.
Under torchrun each rank sketches its own copy of the workload (independent
problems, no collective on the data path): weak scaling; with --split the
ranks share one problem instead (A split by columns for the left sketch, by
rows for the right, S regenerated on every rank, no data exchange): strong
scaling.

The C2 line also carries the metric's other legs: `vs_fp32` (the same step in
the plain FP32 form, and both forms' errors against FP64), `serve` (a
shortened C5 request stream: p50/p99 latency, served TFLOP/s, both forms) and
`roofline.generator_floor_ms`.  `cpu_baseline` and --impl reference time the
oracle on the same sample: whole rows of Y, each against every column.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (m, n, k, dists, side)
    "C2": (1 << 20, 512, 2048, (1, 0), "left"),
    "C1": (4096, 256, 64, (0,), "left"),
    "C3": (65536, 16384, 256, (0,), "right"),
    "C4": (None, None, None, (0, 1), "batch"),
    "C5": (None, None, None, (0, 1), "serve"),
    "NYS": (50000, 50000, None, (0,), "nystrom"),
}
DIST_NAME = {0: "gaussian", 1: "rademacher", 2: "uniform"}
METRIC = "fused gen+sketch TFLOP/s and % roofline vs plain FP32; served p50/p99 latency"
L2_BYTES = 129 * 2**20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def left_kernel_source_sha() -> str | None:
    """Hash of the left sketch's device code (constants, split pass, worker,
    epilogue and MMA code of sk_tc.cu up to the right sketch, the PTX helpers
    of sk_tc.cuh and the generator of sk_rng.cuh), which the committed ncu
    summary records; an edit elsewhere does not invalidate it."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2603_20966_gb300", "csrc")
    try:
        text = open(os.path.join(csrc, "sk_tc.cu")).read()
        helpers = open(os.path.join(csrc, "sk_tc.cuh")).read()
        rng = open(os.path.join(csrc, "sk_rng.cuh")).read()
    except OSError:
        return None
    i0, i1 = text.find("constexpr int BM = 128;"), text.find("// Right sketch Y[m x k]")
    if i0 < 0 or i1 < 0:
        return None
    return hashlib.sha256((text[i0:i1] + helpers + rng).encode()).hexdigest()[:16]


def measured_traffic(dist: int):
    """DRAM bytes of one benchmarked sketch (split pass + sketch kernel) of
    distribution `dist` from the committed ncu summary, or None when the
    left kernel's source changed since the capture."""
    prof = os.path.join(ROOT, "profiles", "k_sketch_bf16x2_left_pair_m2e18.md")
    sha = left_kernel_source_sha()
    try:
        text = open(prof).read()
    except OSError:
        return None
    key = f"traffic_bytes_per_full_sketch_{DIST_NAME[dist]}"
    rec = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line and
               line.split(": ", 1)[0] in ("left_kernel_source_sha256_16", key))
    if sha is None or rec.get("left_kernel_source_sha256_16") != sha:
        return None
    try:
        return float(rec[key])
    except (KeyError, ValueError):
        return None


def max_over_ranks(value: float, device=None) -> float:
    """The largest `value` over all ranks of the default process group (the
    timing rule of the benchmark: the slowest rank defines the step time)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_sample_rows(workload: str, m: int, k: int, side: str) -> int:
    """The CPU oracle's sample of one step, the same in the cpu_baseline leg
    and in --impl reference: whole rows of Y, each against every column of A.
    Left: that many rows of Y = S A, each one S row generated once and used by
    all n columns, as in the full workload.  Right: that many rows of A, all k
    columns of Y each, with S generated once for the call (the full workload
    spreads it over m rows, so the sample is large enough for the product to
    dominate)."""
    if side == "left":
        return min(k, 64)
    return min(m, 1024)


def oracle_sample(m, n, k, dists, a_part, seed, rows, nthreads=None, side="left"):
    """Time the CPU oracle on a sample of Y for each distribution.  Left:
    `rows` rows of Y x the a_part.shape[1] columns of A given.  Right: all k
    columns of Y for the a_part.shape[0] rows of A given.  Returns
    (seconds, useful flops, threads)."""
    import oracle
    nthreads = nthreads or os.cpu_count() or 1
    t0 = time.perf_counter()
    for d in dists:
        if side == "left":
            oracle.apply_left(seed, d, 0, k, a_part, nthreads=nthreads, rows=(0, rows))
        else:
            oracle.apply_right(seed, d, 0, k, a_part, nthreads=nthreads)
    dt = time.perf_counter() - t0
    if side == "left":
        return dt, 2.0 * rows * m * a_part.shape[1] * len(dists), nthreads
    return dt, 2.0 * a_part.shape[0] * n * k * len(dists), nthreads


def generator_floor(dist: int, entries: float, sm_mhz: float, sms: int):
    """Issue-rate floor of the Gaussian sketch kernel, which generation
    bounds: its thread instructions (every role) per generated entry of S,
    from the committed ncu summary of the left kernel (None when that
    kernel's source changed since), over the issue rate of every SM (4
    schedulers x 32 lanes per cycle) -- the kernel's time if it issued an
    instruction on every scheduler in every cycle.  Returns (ms, instructions
    per entry) or None."""
    if dist != 0:
        return None  # sign bits: one Philox word per 32 entries, not separable
    prof = os.path.join(ROOT, "profiles", "k_sketch_bf16x2_left_pair_m2e18.md")
    sha = left_kernel_source_sha()
    try:
        text = open(prof).read()
    except OSError:
        return None
    key = "gaussian_kernel_thread_instructions_per_entry"
    rec = dict(line.split(": ", 1) for line in text.splitlines() if ": " in line and
               line.split(": ", 1)[0] in ("left_kernel_source_sha256_16", key))
    if sha is None or rec.get("left_kernel_source_sha256_16") != sha or key not in rec:
        return None
    ipe = float(rec[key])
    return entries * ipe / (sms * 128 * sm_mhz * 1e6) * 1e3, ipe


def fp32_comparison(P, A, m, n, k, dists, Ys, stream, steps, ncols=32):
    """The metric's comparison: the same left-sketch step in the plain FP32
    form (FP32 FMA on the CUDA cores), timed with CUDA events, and the error
    of both forms against FP64 products of their own S (g for FP32, bf16(g)
    for BF16 split-A, materialized by the library in row blocks of A) over
    `ncols` evenly spaced columns of Y."""
    import numpy as np
    import torch
    dev = A.device
    hs = {d: P.sk_create(7, d, k) for d in dists}  # FP32 is the default form
    Y32 = {d: torch.empty((k, n), dtype=torch.float32, device=dev) for d in dists}

    def step():
        for d in dists:
            P.sk_apply_left(hs[d], A, m, n, n, Y32[d], n, stream)

    step()
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    for d in dists:
        if P.sk_stream_status(hs[d], stream) != 0:
            raise RuntimeError("FP32 comparison: device status")
    cols = torch.from_numpy(np.linspace(0, n - 1, ncols).astype(np.int64)).to(dev)
    A64 = A[:, cols].double()
    block = 1 << 18
    err = {"bf16x2": {}, "fp32": {}}
    for d in dists:
        s = P.sk_get_info(hs[d])["scale"]
        ref32 = torch.zeros((k, ncols), dtype=torch.float64, device=dev)
        ref16 = torch.zeros((k, ncols), dtype=torch.float64, device=dev)
        for c0 in range(0, m, block):
            w = min(block, m - c0)
            S = torch.empty((k, w), dtype=torch.float32, device=dev)
            P.sk_materialize(hs[d], 0, c0, k, w, P.SK_FP32, 0, S, w, stream)
            ref32 += S.double() @ A64[c0:c0 + w]
            Sb = torch.empty((k, w), dtype=torch.bfloat16, device=dev)
            P.sk_materialize(hs[d], 0, c0, k, w, P.SK_BF16X2, 0, Sb, w, stream)
            ref16 += Sb.double() @ A64[c0:c0 + w]
            del S, Sb
        ref32 *= s
        ref16 *= s
        name = DIST_NAME[d]
        err["fp32"][name] = float((Y32[d][:, cols].double() - ref32).norm() / ref32.norm())
        err["bf16x2"][name] = float((Ys[d][:, cols].double() - ref16).norm() / ref16.norm())
        del ref32, ref16
    for d in dists:
        P.sk_destroy(hs[d])
    del Y32, A64
    return ms, err


def run_reference(args):
    """--impl reference: the CPU oracle timed on a bounded sample per step."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import torch

    from paper_2603_20966_gb300.workloads import gaussian_matrix
    m, n, k, dists, side = WORKLOADS[args.workload]
    if side == "nystrom":  # the pair's first (dominant) product, B = A Omega, r = 500
        k, side = 500, "right"
    if side not in ("left", "right"):
        print(json.dumps({"impl": "reference", "unavailable":
                          f"workload {args.workload} has no CPU oracle leg (batch/serving)"}))
        return 0
    rows = cpu_sample_rows(args.workload, m, k, side)
    if side == "left":
        a_part = gaussian_matrix(m, n, 1, device="cpu").numpy()
        what = f"{rows} of {k} rows x all {n} columns of Y"
    else:
        a_part = gaussian_matrix(rows, n, 1, device="cpu").numpy()
        what = f"{rows} of {m} rows x all {k} columns of Y"
    for _ in range(args.warmup):
        oracle_sample(m, n, k, dists, a_part, 7, rows, side=side)
    tot, flops, threads = 0.0, 0.0, 1
    for _ in range(args.steps):
        dt, fl, threads = oracle_sample(m, n, k, dists, a_part, 7, rows, side=side)
        tot += dt
        flops += fl
    value = flops / tot / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{args.workload} {side} sketch A {m}x{n} k={k} "
                   f"dists={[DIST_NAME[d] for d in dists]}", "m": m, "n": n, "k": k},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": f"{what} per distribution per step (FP64 accumulation); "
                                   "the rate of whole rows, not extrapolated"},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """C4: 256 independent left sketches (m log-uniform in [1024, 65536], n
    uniform in [32, 512], k = 2n, distribution by a per-problem coin) in one
    persistent launch, BF16 split-A form, autotuned, graph-captured."""
    import torch

    import paper_2603_20966_gb300 as P
    from paper_2603_20966_gb300.workloads import batched_problems, gaussian_matrix

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
    probs = batched_problems(256, seed=1000 + 1000 * rank)
    stream = torch.cuda.Stream(dev)
    data = []
    b = P.sk_batch_create()
    flops = 0.0
    for i, pr in enumerate(probs):
        lda = (pr.n + 3) // 4 * 4
        A = torch.zeros((pr.m, lda), device=dev)
        A[:, :pr.n] = gaussian_matrix(pr.m, pr.n, 5000 + i, device=dev)
        Y = torch.empty((pr.k, lda), device=dev)
        h = P.sk_create(pr.seed, pr.dist, pr.k)
        P.sk_set_precision(h, P.SK_BF16X2)
        P.sk_batch_add(b, h, A, pr.m, pr.n, lda, Y, lda)
        data.append((h, A, Y))
        flops += 2.0 * pr.k * pr.m * pr.n
    torch.cuda.synchronize(dev)
    P.sk_batch_tune(b, stream)
    chosen = P.sk_batch_config(b)
    for _ in range(args.warmup):
        P.sk_batch_run(b, stream)
    st = P.sk_batch_status(b, stream)
    if st != 0:
        raise RuntimeError(f"batch status: {P.status_string(st)}")
    clocks = ClockSampler(local)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    launches0 = P.sk_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        P.sk_batch_run(b, stream)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    launches = P.sk_launch_count() - launches0
    if P.sk_batch_status(b, stream) != 0:
        raise RuntimeError("batch status after timing")
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    step_ms = ms / args.steps
    pk, pk_kind = peaks()
    value = world * flops * args.steps / (ms * 1e-3) / 1e12
    roof = {"bound": "tensor", "achieved": 2 * flops / (step_ms * 1e-3) / 1e12,
            "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "peak_kind": f"{pk_kind} bf16 burst",
            "note": "achieved counts both split-A passes over the whole batch step (two "
                    "launches: persistent sketch + batched reduce)", "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    P.sk_batch_destroy(b)
    for h, _, _ in data:
        P.sk_destroy(h)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x2",
            "data": "synthetic",
            "config": {"workload": "C4 batch of 256 left sketches, m log-uniform [1024, 65536], "
                                   "n uniform [32, 512], k = 2n, mixed Gaussian/Rademacher",
                       "problems": 256, "useful_tflop_per_step": flops / 1e12,
                       "autotuned": chosen, "form": "bf16x2",
                       "l2": "inputs larger than L2 (A total "
                             f"{sum(p.m * p.n for p in probs) * 4 / 2**30:.2f} GiB)",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk, "e2e": None, "gpu_launches": int(launches), "roofline": roof,
            "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    return 0


def _serve_stream(P, srv, reqs, hs, src_ptr, src_ld, fetch=None):
    """Submit `reqs` at their arrival times (busy-waiting on the host clock)
    and wait until every one has finished.  Returns (wall seconds from the
    first submission to the last completion, max submission lateness s)."""
    import torch
    tickets = []
    late = 0.0
    done = threading.Event()
    errors = []

    def collect():
        # fetch results in submission order (e2e leg): Y to pinned host memory
        i = 0
        while i < len(reqs):
            if i >= len(tickets):
                time.sleep(0.0002)
                continue
            r, t = reqs[i], tickets[i]
            st, _ = P.sk_server_wait(srv, t, 120.0)
            if st != 0:
                errors.append(P.status_string(st))
                break
            P.sk_server_fetch(srv, t, fetch, r.prob.n)
            i += 1
        done.set()

    th = None
    if fetch is not None:
        th = threading.Thread(target=collect, daemon=True)
        th.start()
    t0 = time.perf_counter()
    for i, r in enumerate(reqs):
        target = t0 + r.arrival_s
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            if target - now > 0.002:
                time.sleep(0.001)
        late = max(late, time.perf_counter() - target)
        p = r.prob
        t = P.sk_server_submit(srv, hs[i], src_ptr + 4 * r.row0 * src_ld, p.m, p.n, src_ld)
        if fetch is None:
            P.sk_server_release(srv, t)  # results dropped when they finish
        tickets.append(t)
    deadline = time.perf_counter() + 180.0
    if th is not None:
        done.wait(timeout=180.0)
        if errors or not done.is_set():
            raise RuntimeError(f"serving e2e leg failed: {errors or 'timeout'}")
    else:
        last, t_last = -1, time.perf_counter()
        while time.perf_counter() < deadline:
            s = P.sk_server_stats_get(srv)
            done_n = s["completed"] + s["failed"]
            if done_n >= len(reqs):
                break
            if done_n != last:
                last, t_last = done_n, time.perf_counter()
            elif time.perf_counter() - t_last > 60.0:
                raise RuntimeError(f"serving stream made no progress for 60 s: {s}")
            time.sleep(0.002)
    wall = time.perf_counter() - t0
    s = P.sk_server_stats_get(srv)
    if s["failed"] or s["completed"] < len(reqs):
        raise RuntimeError(f"serving run incomplete: {s}")
    return wall, late


def serve_forms(P, reqs, forms, src, src_host, src_ld, warmup, world, clocks=None,
                e2e_leg=False):
    """Run the request stream `reqs` through a server once per form (name,
    sk_precision) with a 120 GB budget.  Returns ({form: latency and
    throughput figures}, clock record of the first form, end-to-end record
    or None, kernel launches)."""
    import torch
    budget = 120 * 10**9
    out, clk, e2e, launches = {}, None, None, 0
    for fi, (name, form) in enumerate(forms):
        hs = []
        for r in reqs:
            h = P.sk_create(r.prob.seed, r.prob.dist, r.prob.k)
            if form != P.SK_FP32:
                P.sk_set_precision(h, form)
            hs.append(h)
        srv = P.sk_server_create(budget, 4096)
        try:
            # warm-up: the first requests once, all at time zero
            warm = reqs[:max(3, warmup) * 10]
            _serve_stream(P, srv, [type(r)(0.0, r.prob, r.row0) for r in warm], hs,
                          src.data_ptr(), src_ld)
            P.sk_server_reset_stats(srv)
            if world > 1:
                import torch.distributed as tdist
                tdist.barrier()
            if fi == 0 and clocks is not None:
                clocks.start()
            l0 = P.sk_launch_count()
            wall, late = _serve_stream(P, srv, reqs, hs, src.data_ptr(), src_ld)
            launches += P.sk_launch_count() - l0
            if fi == 0 and clocks is not None:
                clk = clocks.stop()
            st = P.sk_server_stats_get(srv)
            out[name] = {"p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
                         "mean_ms": st["mean_ms"], "max_ms": st["max_ms"],
                         "mean_wait_ms": st["mean_wait_ms"],
                         "served_tflops": st["flops"] / wall / 1e12,
                         "wall_s": wall, "steps": st["steps"],
                         "mean_requests_per_step": len(reqs) / max(1, st["steps"]),
                         "max_step_requests": st["max_step_requests"],
                         "peak_pool_gb": st["peak_bytes"] / 1e9,
                         "max_submit_lateness_ms": late * 1e3}
            if fi == 0 and e2e_leg:
                # end to end: sources in pinned host memory (copied in at
                # admission), every Y fetched back to pinned host memory
                P.sk_server_reset_stats(srv)
                y_host = torch.empty((1024, 512), dtype=torch.float32, pin_memory=True)
                wall_e, _ = _serve_stream(P, srv, reqs, hs, src_host.data_ptr(), src_ld,
                                          fetch=y_host)
                st = P.sk_server_stats_get(srv)
                e2e = {"value": st["flops"] / wall_e / 1e12, "unit": "TFLOP/s",
                       "h2d_bytes_per_step": sum(4 * r.prob.m * r.prob.n for r in reqs),
                       "d2h_bytes_per_step": sum(4 * r.prob.k * r.prob.n for r in reqs),
                       "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "wall_s": wall_e,
                       "step": f"the whole {len(reqs)}-request stream from pinned host "
                               "sources, results fetched to pinned host memory"}
        finally:
            P.sk_server_destroy(srv)
            for h in hs:
                P.sk_destroy(h)
    return out, clk, e2e, launches


def serve_source(dev, rank, pinned=True):
    """The load generator's source rows (every request reads a window of
    them): 2^18 x 512 N(0,1) on the device, and a pinned host copy."""
    import torch
    from paper_2603_20966_gb300.workloads import gaussian_matrix
    src_rows, src_ld = 1 << 18, 512
    src = gaussian_matrix(src_rows, src_ld, 77 + rank, device=dev)
    src_host = None
    if pinned:
        src_host = torch.empty((src_rows, src_ld), dtype=torch.float32, pin_memory=True)
        src_host.copy_(src)
    torch.cuda.synchronize(dev)
    return src, src_host, src_ld


def run_serve(args):
    """C5: a Poisson stream of left-sketch requests (2000/s, m log-uniform in
    [1024, 2^18], n uniform in [32, 512], k = 2n) through the request server
    with a 120 GB budget; BF16 split-A and plain FP32 forms; p50/p99 latency
    (arrival to Y ready) and served useful TFLOP/s."""
    import torch

    import paper_2603_20966_gb300 as P
    from paper_2603_20966_gb300.workloads import serving_requests

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
    count = args.serve_requests
    reqs = serving_requests(count, seed=3000 + 1000 * rank)
    src, src_host, src_ld = serve_source(dev, rank)
    clocks = ClockSampler(local)
    out, clk, e2e, launches = serve_forms(
        P, reqs, [("bf16x2", P.SK_BF16X2), ("fp32", P.SK_FP32)], src, src_host, src_ld,
        args.warmup, world, clocks=clocks, e2e_leg=not args.no_e2e)
    flops = sum(2.0 * r.prob.k * r.prob.m * r.prob.n for r in reqs)
    offered = flops / reqs[-1].arrival_s / 1e12
    if rank == 0:
        b = out["bf16x2"]
        line = {
            "metric": METRIC, "value": b["served_tflops"] * world, "unit": "TFLOP/s",
            "n_gpus": world, "steps": count, "warmup": args.warmup,
            "ms_per_step": b["mean_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16x2", "data": "synthetic",
            "config": {"workload": f"C5 serving: Poisson stream of {count} left-sketch "
                                   "requests at 2000/s, m log-uniform [1024, 2^18], n uniform "
                                   "[32, 512], k = 2n, mixed Gaussian/Rademacher, 120 GB budget",
                       "offered_tflops": offered, "useful_tflop": flops / 1e12,
                       "step": "one step = one request; ms_per_step = mean latency",
                       "l2": "request windows drawn from a 512 MiB source, larger than L2",
                       "parallelism": f"replicas x{world}"},
            "latency_ms": {"bf16x2": {"p50": b["p50_ms"], "p99": b["p99_ms"]},
                           "fp32": {"p50": out["fp32"]["p50_ms"], "p99": out["fp32"]["p99_ms"]}},
            "forms": out, "clocks": clk, "e2e": e2e, "gpu_launches": int(launches),
            "roofline": None, "cpu_baseline": None,
        }
        print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as tdist

    import paper_2603_20966_gb300 as P
    from paper_2603_20966_gb300.workloads import gaussian_matrix

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        tdist.init_process_group("nccl", device_id=dev)
    m, n, k, dists, side = WORKLOADS[args.workload]
    if args.rows is not None:  # a smaller case of the same workload (profiling captures)
        m = args.rows
    if args.dists is not None:
        dists = tuple(int(x) for x in args.dists.split(","))
    form = {"fp32": P.SK_FP32, "bf16x2": P.SK_BF16X2, "fp8": P.SK_FP8E4M3}[args.form]
    if form == P.SK_FP8E4M3 and side != "right":
        raise SystemExit("the FP8 form is the right sketch only (workload C3)")
    stream = torch.cuda.current_stream(dev)
    apply = P.sk_apply_left if side == "left" else P.sk_apply_right
    apply_host = P.sk_apply_left_host if side == "left" else P.sk_apply_right_host
    yshape = (k, n) if side == "left" else (m, k)

    if args.workload == "C3":
        from paper_2603_20966_gb300.workloads import lowrank_plus_noise
        A = lowrank_plus_noise(m, n, device=dev, seeds=(11 + 3 * rank, 12 + 3 * rank,
                                                        13 + 3 * rank))
    else:
        A = gaussian_matrix(m, n, 1 + rank, device=dev)
    Ys = {d: torch.empty(yshape, dtype=torch.float32, device=dev) for d in dists}
    hs = {}
    for d in dists:
        hs[d] = P.sk_create(7, d, k)
        P.sk_set_precision(hs[d], form)
    # what this rank computes: the whole problem (replicas), or with --split
    # its block of one problem shared by all ranks (the paper's Case 1: A split
    # by columns for the left sketch, by rows for the right; every rank
    # regenerates the same S; no data exchange)
    A_run, m_run, n_run, lda_run = A, m, n, n
    Y_run = dict(Ys)
    part = None
    if args.split:
        from paper_2603_20966_gb300.partition import left_column_ranges, right_row_ranges
        if side == "left":
            c0, c1 = left_column_ranges(n, world)[rank]
            A_run, n_run = A[:, c0:c1], c1 - c0
            Y_run = {d: Ys[d][:, c0:c1] for d in dists}
            part = {"columns": [c0, c1]}
        else:
            r0, r1 = right_row_ranges(m, world)[rank]
            A_run, m_run = A[r0:r1], r1 - r0
            Y_run = {d: Ys[d][r0:r1] for d in dists}
            part = {"rows": [r0, r1]}
    ldy_run = yshape[1]

    def step():
        for d in dists:
            apply(hs[d], A_run, m_run, n_run, lda_run, Y_run[d], ldy_run, stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    for d in dists:
        st = P.sk_stream_status(hs[d], stream)
        if st != 0:
            raise RuntimeError(f"device status after warm-up: {P.status_string(st)}")

    # per-launch events of the fused kernel, recorded by the library hook
    nl = args.steps * len(dists)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(nl)]
    for a, b in ev:  # create the underlying events before handing them out
        a.record(stream)
        b.record(stream)
    torch.cuda.synchronize(dev)

    clocks = ClockSampler(local)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    launches0 = P.sk_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_stop = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    i = 0
    for _ in range(args.steps):
        for d in dists:
            P.sk_profile_events(hs[d], ev[i][0], ev[i][1])
            apply(hs[d], A_run, m_run, n_run, lda_run, Y_run[d], ldy_run, stream)
            i += 1
    t_stop.record(stream)
    torch.cuda.synchronize(dev)
    launches = P.sk_launch_count() - launches0
    if world > 1:
        tdist.barrier()
    clk = clocks.stop()
    for d in dists:
        P.sk_profile_events(hs[d], None, None)
        st = P.sk_stream_status(hs[d], stream)
        if st != 0:
            raise RuntimeError(f"device status after timing: {P.status_string(st)}")
    ms = max_over_ranks(t_start.elapsed_time(t_stop), dev)
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    flops_per_sketch = 2.0 * k * m_run * n_run  # this rank's sketch (or block of one)
    flops_step = flops_per_sketch * len(dists)
    # whole job: N replicas of the problem, or one problem split over N ranks
    job_flops_step = (2.0 * k * m * n * len(dists)) if args.split else world * flops_step
    value = job_flops_step * args.steps / (ms * 1e-3) / 1e12

    pk, pk_kind = peaks()
    avg_kernel_s = statistics.mean(kernel_ms) * 1e-3
    if form == P.SK_FP32:
        # FP32 FMA pipe: 152 SMs x 128 lanes x 2 flop x max SM clock
        peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": flops_per_sketch / avg_kernel_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_kind": "derived: 152 SM x 128 FP32 lanes x 2 x "
                                                "max SM clock"}
    elif side == "right" and form == P.SK_FP8E4M3:
        # the timed kernel is the FP8 sketch: E4M3 A read once, Y written once
        algo_bytes = 1.0 * m * n + 4.0 * m * k
        peak = pk["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": algo_bytes / avg_kernel_s / 1e9, "peak": peak,
                "unit": "GB/s", "peak_kind": f"{pk_kind} copy bandwidth",
                "note": "timed kernel = the FP8 sketch; achieved = (E4M3 A bytes + Y bytes) / "
                        "its time; the step also runs the row quantizer (FP32 A read once, "
                        "codes written once)"}
    elif side == "right":
        # HBM-bound: A read once, Y written once
        algo_bytes = 4.0 * m_run * n_run + 4.0 * m_run * k
        peak = pk["hbm_gbs"]
        roof = {"bound": "hbm", "achieved": algo_bytes / avg_kernel_s / 1e9, "peak": peak,
                "unit": "GB/s", "peak_kind": f"{pk_kind} copy bandwidth",
                "note": "achieved = (A bytes + Y bytes) / kernel time"}
    else:
        mma = 2 * flops_per_sketch  # split-A: two BF16 MMA passes
        peak = pk["bf16_tflops"]
        roof = {"bound": "tensor", "achieved": mma / avg_kernel_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_kind": f"{pk_kind} bf16 burst",
                "note": "achieved counts both split-A MMA passes (4 k m n flop per sketch)"}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if form == P.SK_BF16X2 and side == "left" and args.rows is None:
        tr = [measured_traffic(d) for d in dists]
        roof["traffic"] = None if any(t is None for t in tr) else sum(tr) / len(tr)
        if roof["traffic"] is not None:
            roof["traffic_note"] = ("DRAM bytes per sketch (split pass + sketch kernel, average "
                                    "over the distributions) from the committed ncu summary")
    else:
        roof["traffic"] = None
    roof["kernel_ms_by_dist"] = {DIST_NAME[d]: statistics.mean(kernel_ms[j::len(dists)])
                                 for j, d in enumerate(dists)}

    fp8 = None
    if form == P.SK_FP8E4M3 and not args.split:
        # a resident quantized A (quantized once, outside the timed region)
        ldq = (n + 15) // 16 * 16
        Aq = torch.empty((m, ldq), dtype=torch.uint8, device=dev)
        ex = torch.empty((m,), dtype=torch.int32, device=dev)
        P.sk_quantize_e4m3(A, m, n, n, Aq, ldq, ex, stream)
        for _ in range(2):
            for d in dists:
                P.sk_apply_right_e4m3(hs[d], Aq, ex, m, n, ldq, Ys[d], yshape[1], stream)
        q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        q0.record(stream)
        for _ in range(args.steps):
            for d in dists:
                P.sk_apply_right_e4m3(hs[d], Aq, ex, m, n, ldq, Ys[d], yshape[1], stream)
        q1.record(stream)
        torch.cuda.synchronize(dev)
        qms = q0.elapsed_time(q1) / args.steps
        fp8 = {"resident_e4m3_a": {"ms_per_step": qms,
                                   "tflops": flops_step / (qms * 1e-3) / 1e12,
                                   "hbm_gbs": len(dists) * (m * n + 4.0 * m * k) / (qms * 1e-3) / 1e9},
               "note": "resident: A quantized once (sk_quantize_e4m3) and sketched by "
                       "sk_apply_right_e4m3 each step; error vs the exact product is reported "
                       "by tests/test_gpu_fp8.py (about 3-4 %)"}
        del Aq, ex

    # generate versus communicate (Sec. 6.2): the same kernel reading a
    # materialized BF16 S from HBM instead of generating it
    ablation = None
    if form == P.SK_BF16X2 and side == "left" and not args.no_ablation and not args.split:
        lds = (m + 15) // 16 * 16
        ablation = {"S_bytes": 2 * k * lds, "fused_kernel_ms": {}, "stored_kernel_ms": {},
                    "materialize_ms": {}, "identical_to_fused": {},
                    "note": "stored = sk_apply_left_stored reading S (materialized once by "
                            "sk_materialize, BF16) by TMA in place of generating it; "
                            "kernel times bracket the split pass and the sketch kernel, as "
                            "for the fused path"}
        for j, d in enumerate(dists):
            S = torch.zeros((k, lds), dtype=torch.bfloat16, device=dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            P.sk_materialize(hs[d], 0, 0, k, m, P.SK_BF16X2, 0, S, lds, stream)
            e1.record(stream)
            Yst = torch.empty(yshape, dtype=torch.float32, device=dev)
            reps = max(3, min(args.steps, 10))
            sev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(reps)]
            for a, b in sev:
                a.record(stream)
                b.record(stream)
            P.sk_apply_left_stored(hs[d], S, lds, A, m, n, n, Yst, yshape[1], stream)  # warm
            for a, b in sev:
                P.sk_profile_events(hs[d], a, b)
                P.sk_apply_left_stored(hs[d], S, lds, A, m, n, n, Yst, yshape[1], stream)
            P.sk_profile_events(hs[d], None, None)
            torch.cuda.synchronize(dev)
            st = P.sk_stream_status(hs[d], stream)
            if st != 0:
                raise RuntimeError(f"device status after the stored-S sketch: "
                                   f"{P.status_string(st)}")
            name = DIST_NAME[d]
            ablation["materialize_ms"][name] = e0.elapsed_time(e1)
            ablation["stored_kernel_ms"][name] = statistics.mean(a.elapsed_time(b)
                                                                 for a, b in sev)
            ablation["fused_kernel_ms"][name] = roof["kernel_ms_by_dist"][name]
            ablation["identical_to_fused"][name] = bool(torch.equal(Yst, Ys[d]))
            del S, Yst

    # the metric's other legs: the same step in plain FP32, with the error of
    # both forms against FP64 measured in this run; the served latencies of a
    # shortened C5 stream; the generator's issue-rate floor
    vs_fp32 = None
    if (form == P.SK_BF16X2 and side == "left" and args.rows is None and not args.no_fp32 and
            not args.split):
        fms, ferr = fp32_comparison(P, A, m, n, k, dists, Ys, stream, args.fp32_steps)
        fp32_tflops = world * flops_step / (fms * 1e-3) / 1e12
        vs_fp32 = {"fp32_tflops": fp32_tflops, "fp32_ms_per_step": fms,
                   "bf16x2_over_fp32": value / fp32_tflops,
                   "fp32_steps": args.fp32_steps, "err_vs_fp64": ferr,
                   "err_note": "relative Frobenius error of Y over 32 evenly spaced columns "
                               "against FP64 products with each form's own S (g for FP32, "
                               "bf16(g) for BF16 split-A) materialized by the library; "
                               "tolerance 1e-5",
                   "fp32_form": "FP32 FMA on the CUDA cores, S generated in shared memory"}
    if roof.get("bound") == "tensor":
        clk_mhz = (clk or {}).get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        floors = {}
        for d in dists:
            f = generator_floor(d, float(k) * float(m), clk_mhz, sms)
            if f is not None:
                floors[DIST_NAME[d]] = {"ms": f[0], "thread_instructions_per_entry": f[1]}
        roof["generator_floor_ms"] = ({nm: v["ms"] for nm, v in floors.items()}
                                      if floors else None)
        if floors:
            roof["generator_floor_note"] = (
                "entries x the Gaussian kernel's thread instructions per generated entry "
                "(every role; committed ncu summary of this kernel source) / (SMs x 128 issue "
                f"lanes x median SM clock): its time at full issue, {floors}")
    serve = None
    if (args.workload == "C2" and args.rows is None and args.serve_leg_requests > 0 and
            not args.split):
        from paper_2603_20966_gb300.workloads import serving_requests
        reqs = serving_requests(args.serve_leg_requests, seed=3000 + 1000 * rank)
        src, _, src_ld = serve_source(dev, rank, pinned=False)
        sout, _, _, _ = serve_forms(P, reqs, [("bf16x2", P.SK_BF16X2), ("fp32", P.SK_FP32)],
                                    src, None, src_ld, 3, world)
        del src
        fl = sum(2.0 * r.prob.k * r.prob.m * r.prob.n for r in reqs)
        serve = {"requests": len(reqs), "rate_per_s": 2000.0,
                 "offered_tflops": fl / reqs[-1].arrival_s / 1e12,
                 "latency_ms": {f: {"p50": sout[f]["p50_ms"], "p99": sout[f]["p99_ms"]}
                                for f in sout},
                 "served_tflops": {f: sout[f]["served_tflops"] for f in sout},
                 "forms": sout,
                 "note": f"shortened C5 stream: the first {len(reqs)} of its 20000 requests "
                         "(Poisson arrivals at 2000/s, m log-uniform [1024, 2^18], n uniform "
                         "[32, 512], k = 2n, 120 GB budget); latency = arrival to Y ready; "
                         "the full stream is bench.py --workload C5"}

    # end to end through the host-buffer entry points
    e2e = None
    if not args.no_e2e:
        # this rank's block of A in pinned host memory, its block of Y back
        A_host = torch.empty((m_run, n_run), dtype=torch.float32, pin_memory=True)
        A_host.copy_(A_run)
        yb = (k, n_run) if side == "left" else (m_run, k)
        Y_host = {d: torch.empty(yb, dtype=torch.float32, pin_memory=True) for d in dists}

        def e2e_step():
            for d in dists:
                apply_host(hs[d], A_host, m_run, n_run, n_run, Y_host[d], yb[1], stream)

        for _ in range(max(1, min(args.warmup, 2))):
            e2e_step()
        if world > 1:
            tdist.barrier()
        e_steps = max(1, min(args.steps, 5))
        t0 = time.perf_counter()
        for _ in range(e_steps):
            e2e_step()
        dt = max_over_ranks(time.perf_counter() - t0, dev)
        e2e = {"value": job_flops_step * e_steps / dt / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": len(dists) * m_run * n_run * 4,
               "d2h_bytes_per_step": len(dists) * yb[0] * yb[1] * 4, "steps": e_steps,
               "ms_per_step": dt / e_steps * 1e3}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rows = cpu_sample_rows(args.workload, m, k, side)
        if side == "left":
            a_part = A.cpu().numpy()
            what = f"{rows} of {k} rows x all {n} columns of Y"
        else:
            idx = np.linspace(0, m - 1, rows).astype(np.int64)
            a_part = A[torch.from_numpy(idx).to(dev)].cpu().numpy()
            what = f"{rows} of {m} rows x all {k} columns of Y"
        dt, fl, threads = oracle_sample(m, n, k, dists, a_part, 7, rows, side=side)
        cpu = {"value": fl / dt / 1e12, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
               "sample": f"{what} for each of {[DIST_NAME[d] for d in dists]} "
                         f"(FP64 accumulation), {dt:.1f} s; whole rows, each S row generated "
                         f"once for all columns as in the full workload (the --impl "
                         f"reference sample); the rate of the sample, not extrapolated"}
        del a_part

    for d in dists:
        P.sk_destroy(hs[d])
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "strong" if args.split else "weak",
            "vs_baseline": None,
            "dtype": {"fp32": "f32", "bf16x2": "bf16x2", "fp8": "e4m3"}[args.form],
            "data": "synthetic",
            "config": {"workload": f"{args.workload} {side} sketch A {m}x{n} FP32 "
                                   f"{'U V^T + 1e-3 E' if args.workload == 'C3' else 'N(0,1)'}, "
                                   f"k={k}, S {[DIST_NAME[d] for d in dists]} Philox4x32-10 "
                                   f"seed 7",
                       "m": m, "n": n, "k": k, "form": args.form,
                       "l2": f"inputs larger than L2 (A {m * n * 4 / 2**30:.2f} GiB)",
                       "parallelism": (f"split x{world}: one problem, A by "
                                       f"{'columns' if side == 'left' else 'rows'}, S "
                                       f"regenerated on every rank, no data exchange"
                                       if args.split else f"replicas x{world}")},
            "clocks": clk, "e2e": e2e, "gpu_launches": int(launches), "roofline": roof,
            "cpu_baseline": cpu,
        }
        if part is not None:
            line["config"]["rank0_block"] = part
        if vs_fp32 is not None:
            line["vs_fp32"] = vs_fp32
        if serve is not None:
            line["serve"] = serve
        if fp8 is not None:
            line["fp8"] = fp8
        if ablation is not None:
            line["gen_vs_comm"] = ablation
        print(json.dumps(line), flush=True)
    if world > 1:
        tdist.destroy_process_group()
    return 0


def run_nystrom(args):
    """NYS: the Nystrom pair of the paper's Alg. 2 (B = A Omega, C = Omega^T B,
    the same Gaussian Omega regenerated by both products) on a 50000 x 50000
    RBF kernel matrix, r = 500 and r = 5000 (the paper's ranks), BF16 split-A
    form.  A step is one r; `value` is the r = 500 line, the r = 5000 figures
    ride along in `ranks`."""
    import torch

    import paper_2603_20966_gb300 as P
    from paper_2603_20966_gb300.workloads import rbf_kernel_matrix

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl", device_id=dev)
    n = WORKLOADS["NYS"][0] if args.rows is None else args.rows
    A = rbf_kernel_matrix(n, seed=21 + rank, device=dev)
    stream = torch.cuda.Stream(dev)
    pk, pk_kind = peaks()
    ranks = {}
    clocks = ClockSampler(local)
    clk = None
    launches = 0
    for r in (500, 5000):
        ld = (r + 3) // 4 * 4
        B = torch.empty((n, ld), dtype=torch.float32, device=dev)
        C = torch.empty((r, ld), dtype=torch.float32, device=dev)
        h = P.sk_create(7, 0, r)
        P.sk_set_precision(h, P.SK_BF16X2)
        steps = args.steps if r == 500 else max(1, min(args.steps, 10))
        for _ in range(args.warmup):
            P.sk_nystrom(h, A, n, n, B, ld, C, ld, stream)
        if P.sk_stream_status(h, stream) != 0:
            raise RuntimeError("nystrom status")
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize(dev)
        if r == 500:
            clocks.start()
            launches0 = P.sk_launch_count()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            P.sk_nystrom(h, A, n, n, B, ld, C, ld, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if r == 500:
            clk = clocks.stop()
            launches = P.sk_launch_count() - launches0
        if P.sk_stream_status(h, stream) != 0:
            raise RuntimeError("nystrom status after timing")
        ms = max_over_ranks(e0.elapsed_time(e1), dev) / steps
        flops = 2.0 * n * n * r + 2.0 * r * n * r
        # symmetry of C = Omega^T A Omega for a symmetric A (a cheap sanity check)
        Cs = C[:, :r].double()
        asym = float((Cs - Cs.t()).norm() / Cs.norm())
        ranks[r] = {"ms_per_step": ms, "tflops": world * flops / (ms * 1e-3) / 1e12,
                    "useful_tflop_per_step": flops / 1e12, "c_asymmetry": asym,
                    "steps": steps}
        P.sk_destroy(h)
        del B, C
    r5 = ranks[500]
    # both products on the tensor cores: 2 passes x (2 n^2 r + 2 r^2 n) flop
    roof = {"bound": "tensor", "achieved": 2 * r5["useful_tflop_per_step"] / (r5["ms_per_step"] * 1e-3),
            "peak": pk["bf16_tflops"], "unit": "TFLOP/s", "peak_kind": f"{pk_kind} bf16 burst",
            "note": "whole step (right sketch B = A Omega, then left sketch C = Omega^T B), both "
                    "split-A passes counted", "traffic": None}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if rank == 0:
        line = {
            "metric": METRIC, "value": r5["tflops"], "unit": "TFLOP/s", "n_gpus": world,
            "steps": r5["steps"], "warmup": args.warmup, "ms_per_step": r5["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16x2",
            "data": "synthetic",
            "config": {"workload": f"NYS Nystrom pair of a {n}x{n} RBF kernel matrix (50000 "
                                   "N(0, I_64) points, sigma^2 = |X|_F^2 / n), Gaussian Omega, "
                                   "r = 500 (line) and 5000 (ranks)",
                       "n": n, "r": 500, "form": "bf16x2",
                       "l2": f"inputs larger than L2 (A {n * n * 4 / 2**30:.2f} GiB)",
                       "parallelism": f"replicas x{world}"},
            "clocks": clk, "e2e": None, "gpu_launches": int(launches), "roofline": roof,
            "cpu_baseline": None, "ranks": ranks,
        }
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="bf16x2", choices=["fp32", "bf16x2", "fp8"])
    ap.add_argument("--workload", default="C2", choices=sorted(WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ablation", action="store_true",
                    help="skip the stored-S (generate versus communicate) comparison")
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--serve-leg-requests", type=int, default=4000,
                    help="requests of the shortened C5 stream in the C2 line (0: none)")
    ap.add_argument("--no-fp32", action="store_true",
                    help="skip the FP32 comparison leg of the C2 line")
    ap.add_argument("--fp32-steps", type=int, default=3)
    ap.add_argument("--split", action="store_true",
                    help="C1-C3 under torchrun: one problem split over the ranks (A by columns "
                         "for the left sketch, by rows for the right; strong scaling) instead "
                         "of one problem per rank")
    ap.add_argument("--rows", type=int, default=None,
                    help="rows of A (C1-C3): a smaller case of the workload, for ncu captures")
    ap.add_argument("--dists", default=None, help="comma-separated distributions (0 G, 1 R, 2 U)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if WORKLOADS[args.workload][4] == "batch":
        return run_batch(args)
    if WORKLOADS[args.workload][4] == "serve":
        return run_serve(args)
    if WORKLOADS[args.workload][4] == "nystrom":
        return run_nystrom(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
