#!/usr/bin/env python
"""Benchmark of wavelet-tree construction on one GB300 (one JSON line).

A step is one pass of the whole hot path over one batch of synthetic input.
With the default workload, two sequences are each built into a resident
pointerless wavelet tree:
- the text-like sequence: 2^30 uint8 codes over 96 symbols, Zipf 1.0;
- the DNA-like sequence: 2^30 uint8 codes over 4 symbols, uniform.
Each build runs the histogram and node starts, then the fused level passes
or the dd-direct kernels, as the autotuner picks.  Then one batch of 2^16
mixed access/rank/select queries runs against the two trees.  The metric is
built symbols per second.  Inputs are larger than L2, so no flush is needed
between steps.

``--workload batch`` times the batched build instead: 4096 sequences of
log-uniform length in [2^10, 2^22], alphabets {4, 20, 256, 65536}, uniform or
Zipf(1.1), built by one wt_build_batch call per step (one CUDA graph), and
reports its efficiency against the plain single-sequence path.
``--workload serve`` runs the serving loop: Poisson arrivals of build
requests at 70% of the measured batched build throughput, continuous
batching under a 120 GB budget, batches of 2^16 mixed queries against the
resident trees, and reports p50/p99 build and query latency.

``--workload locality`` builds the paper's locality stress inputs (Section 4,
cont and rand): n = 2^30 four-byte codes over sigma = 2^y, y in {4, 6, ...,
14}, each code n / sigma times, in code order (cont) or at random positions
(rand); one line with the whole set's throughput and each input's rate.

``--workload merge`` runs the buffered build of Section 5 on the default
sequences: each built in 2^28-symbol chunks whose partial trees are then
merged (wt_build_chunked), with the merge step's own bandwidth.

``--workload matrix`` builds the wavelet matrices of the default sequences
(the level-wise variant Section 5 names for future work).

``--impl reference`` times the CPU oracle instead (single thread, bounded
sample of the same workload).  Under torchrun every rank builds its own
replica (weak scaling, no collective on the data path); rank 0 prints.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1610_05994_gb300 import inputs  # noqa: E402

METRIC = "wavelet-tree build symbols/sec"
UNIT = "symbols/s"
QUERIES = 1 << 16
# The default workload (text + DNA) is the one the headline metric is quoted
# on; "words" is the large-alphabet single-sequence workload.
WORKLOAD_SETS = {
    "text+dna": [inputs.WORKLOADS["u8-text-2^30-s96-zipf1.0"], inputs.WORKLOADS["u8-dna-2^30-s4"]],
    "words": [inputs.WORKLOADS["u32-words-2^29-s2^20-zipf1.2"]],
}
WORKLOAD_NAMES = {
    "text+dna": "u8 text n=2^30 sigma=96 Zipf(1.0) + u8 DNA n=2^30 sigma=4 uniform + 2^16 mixed queries",
    "words": "u32 word ids n=2^29 sigma=2^20 Zipf(1.2) + 2^16 mixed queries",
}


def config_for(name: str) -> dict:
    seqs = WORKLOAD_SETS[name]
    return {"workload": WORKLOAD_NAMES[name],
            "sequences": [{"name": w.name, "n": w.n, "sigma": w.sigma, "width": w.width,
                           "dist": w.dist + (f"{w.alpha}" if w.dist == "zipf" else "")} for w in seqs],
            "queries_per_step": QUERIES,
            "l2": "inputs (>= 1 GiB each) larger than the 129 MB L2; no flush"}
ORACLE_SAMPLE = {"text+dna": 1 << 28, "words": 1 << 24}     # cpu_baseline: 10-30 s of oracle work
REFERENCE_SAMPLE = {"text+dna": 1 << 26, "words": 1 << 23}  # --impl reference, per step


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(x: float, ws: int) -> float:
    """The largest x over all ranks (x itself with one rank).  The tensor
    lives where the process group's backend wants it (GPU for NCCL)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(x: float, ws: int) -> float:
    """The sum of x over all ranks."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_per_rank: float, ws: int, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank does the same work)."""
    return units_per_rank * ws / (ms * 1e-3)


def barrier(ws: int) -> None:
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# The sources of the level step's kernels (count, scans, rank tables, pass):
# the DRAM traffic recorded in profiles/traffic.json holds while they are
# unchanged.
LEVEL_STEP_SOURCES = ("level.cu", "level_common.cuh", "wt_internal.cuh", "build.cu")


def source_hash() -> str:
    h = hashlib.sha256()
    for f in LEVEL_STEP_SOURCES:
        with open(os.path.join(ROOT, "paper_1610_05994_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


RUN = {"workload": None, "size_log2": None, "variant": 0}  # what this invocation measures


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources for this invocation's workload at
    full size; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != source_hash():
        return None
    if rec.get("workload") != RUN["workload"] or RUN["size_log2"] or RUN["variant"] not in (0, 1):
        return None
    return rec.get("dram_bytes_per_launch")


def make_queries(seqs, sigmas, m, seed):
    """Host arrays of a mixed query batch over the trees (uniform tree, op,
    position; c drawn from the sequence; j within the symbol's count)."""
    rng = np.random.default_rng(seed)
    k = len(seqs)
    tidx = rng.integers(0, k, m).astype(np.uint32)
    op = rng.integers(0, 3, m).astype(np.uint8)
    c = np.zeros(m, np.uint32)
    arg = np.zeros(m, np.uint64)
    for t in range(k):
        sel = np.flatnonzero(tidx == t)
        S = seqs[t]
        n = len(S)
        pos = rng.integers(0, n, len(sel))
        c[sel] = S[pos]
        counts = np.bincount(S[: min(n, 1 << 24)], minlength=sigmas[t]).astype(np.float64) * (n / min(n, 1 << 24))
        i_arg = rng.integers(0, n + 1, len(sel)).astype(np.uint64)
        j_arg = (1 + np.floor(rng.random(len(sel)) * np.maximum(counts[c[sel]] * 0.9, 1))).astype(np.uint64)
        arg[sel] = np.where(op[sel] == 2, j_arg, i_arg)
    return tidx, op, c, arg


def run_reference(args, ws, rank):
    """The CPU oracle as it stands, timed on a bounded sample of the workload."""
    if rank != 0:
        return
    from oracle import oracle as O
    O.build()
    n = REFERENCE_SAMPLE[args.workload]
    seqs = [(w.generate(min(n, w.n)), w.sigma) for w in WORKLOAD_SETS[args.workload]]
    for _ in range(min(args.warmup, 1)):
        O.build_bits(seqs[0][0][: 1 << 20], seqs[0][1])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for S, sigma in seqs:
            O.build_bits(S, sigma)
        times.append(time.perf_counter() - t0)
    sec = statistics.median(times)
    syms = sum(len(S) for S, _ in seqs)
    value = syms / sec
    sample = (f"first {min(n, seqs[0][0].size)} symbols of each sequence of the workload, oracle build_bits "
              f"(level-by-level stable partition), 1 thread, median of {args.steps}")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_of(args.workload), "data": "synthetic", "impl": "reference",
            "config": config_for(args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def dtype_of(workload: str) -> str:
    widths = sorted({w.width for w in WORKLOAD_SETS[workload]})
    return "+".join({1: "u8", 2: "u16", 4: "u32"}[x] for x in widths)


def cpu_baseline_sample(workload: str):
    """The oracle timed once on a bounded prefix of every sequence (10-30 s)."""
    from oracle import oracle as O
    O.build()
    n = ORACLE_SAMPLE[workload]
    seqs = [(w.generate(min(n, w.n)), w.sigma) for w in WORKLOAD_SETS[workload]]
    t0 = time.perf_counter()
    for S, sigma in seqs:
        O.build_bits(S, sigma)
    sec = time.perf_counter() - t0
    syms = sum(len(S) for S, _ in seqs)
    return {"value": syms / sec, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n} symbols of each sequence, oracle build_bits, 1 thread, {sec:.1f} s"}


def run_ours(args, ws, rank, local):
    import torch
    import torch.distributed as dist

    from paper_1610_05994_gb300 import build as B
    from paper_1610_05994_gb300 import wt as W

    torch.cuda.set_device(local)
    B.build_library()
    W.load()
    dev = torch.device("cuda", local)

    wls = WORKLOAD_SETS[args.workload]
    host = [w.generate(min(w.n, 1 << args.size_log2) if args.size_log2 else None) for w in wls]
    sigmas = [w.sigma for w in wls]
    tidx, op, c, arg = make_queries(host, sigmas, QUERIES, 7)
    seq_d = [torch.from_numpy(h).to(dev) for h in host]
    q_d = [torch.from_numpy(x).to(dev) for x in (tidx, op, c, arg)]
    out_d = torch.empty(QUERIES, dtype=torch.uint64, device=dev)
    torch.cuda.synchronize()

    def step(keep):
        trees = [W.Tree.build(S, sigma, variant=args.variant, wait=False) for S, sigma in zip(seq_d, sigmas)]
        W.query_multi(trees, *q_d, out=out_d)
        # release the previous step's trees in stream order (no host wait)
        for t in keep:
            t.free()
        return trees

    keep = []
    for _ in range(args.warmup):
        keep = step(keep)
    for t in keep:
        t.wait()
    barrier(ws)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    W.profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        keep = step(keep)
    e1.record()
    torch.cuda.synchronize()
    barrier(ws)
    stats = W.profile_end()
    clk = clocks.stop()
    for t in keep:
        t.wait()
        t.free()
    keep = []
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, ws)
    syms_rank = sum(h.size for h in host)
    value = job_rate(syms_rank, ws, ms)

    # End to end: the same step through the C ABI from pinned host buffers,
    # copies inside the timed region, query answers read back every step.
    host_p = [torch.from_numpy(h).pin_memory() for h in host]
    q_p = [torch.from_numpy(x).pin_memory() for x in (tidx, op, c, arg)]
    out_p = torch.empty(QUERIES, dtype=torch.uint64).pin_memory()

    def step_e2e(keep):
        trees = [_build_from_host(W, p, sigma, args.variant) for p, sigma in zip(host_p, sigmas)]
        qd = [x.to(dev, non_blocking=True) for x in q_p]
        W.query_multi(trees, *qd, out=out_d)
        out_p.copy_(out_d, non_blocking=True)
        for t in keep:
            t.free()
        return trees

    keep = []
    for _ in range(max(1, args.warmup // 2)):
        keep = step_e2e(keep)
    torch.cuda.synchronize()
    barrier(ws)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record()
    e2e_steps = max(1, min(args.steps, 5))
    for _ in range(e2e_steps):
        keep = step_e2e(keep)
    f1.record()
    torch.cuda.synchronize()
    for t in keep:
        t.wait()
        t.free()
    ms_e2e = reduce_max(f0.elapsed_time(f1) / e2e_steps, ws)
    h2d = sum(h.nbytes for h in host) + sum(x.numel() * x.element_size() for x in q_p)
    d2h = QUERIES * 8

    if rank != 0:
        return
    roofline, kernels, launches = roofline_of(stats, args.steps)
    cpu = None if args.no_cpu_baseline or ws > 1 else cpu_baseline_sample(args.workload)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_of(args.workload), "data": "synthetic",
            "config": dict(config_for(args.workload), parallelism=f"replicas{ws}",
                           variant={0: "auto", 1: "levelwise", 2: "dd", 3: "pairs"}[args.variant],
                           **({"reduced_size_log2": args.size_log2} if args.size_log2 else {})),
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": job_rate(syms_rank, ws, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
            "gpu_launches": launches, "clocks": clk, "kernels": kernels}
    print(json.dumps(line), flush=True)


LOCALITY_N = 1 << 30


def run_locality(args, ws, rank, local):
    """Builds of the cont and rand inputs for every sigma = 2^y: per input W
    untimed and K timed builds (CUDA events), the whole set's symbols over
    the sum of the per-input times, and each input's own rate."""
    import torch

    from paper_1610_05994_gb300 import build as B
    from paper_1610_05994_gb300 import wt as W

    torch.cuda.set_device(local)
    B.build_library()
    W.load()
    dev = torch.device("cuda", local)
    n = LOCALITY_N if not args.size_log2 else min(LOCALITY_N, 1 << args.size_log2)
    per, stats, total_ms, e2e = [], {}, 0.0, None
    clocks = ClockSampler(local)
    clocks.start()
    for y in inputs.LOCALITY_SIZES:
        for kind in ("cont", "rand"):
            sigma = 1 << y
            S = inputs.locality_torch(n, sigma, kind, inputs.SEED_BASE + 100 + y, dev)
            for _ in range(args.warmup):
                W.Tree.build(S, sigma, wait=False).free()
            torch.cuda.synchronize()
            barrier(ws)
            W.profile_begin()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.steps):
                W.Tree.build(S, sigma, wait=False).free()
            e1.record()
            torch.cuda.synchronize()
            st = W.profile_end()
            ms = reduce_max(e0.elapsed_time(e1) / args.steps, ws)
            for k, v in st.items():
                acc = stats.setdefault(k, {"launches": 0, "kernels": 0, "total_ms": 0.0, "alg_bytes": 0.0})
                for f in acc:
                    acc[f] += v[f]
            lp = st.get("level_pass")
            per.append({"sigma": sigma, "kind": kind, "ms_per_build": ms, "symbols_per_s": n / (ms * 1e-3),
                        "level_pass_GBps": lp["alg_bytes"] / lp["total_ms"] / 1e6 if lp else None})
            total_ms += ms
            if y == inputs.LOCALITY_SIZES[-1] and kind == "rand":
                # End to end for this input: the build from a pinned host copy.
                host = S.cpu().pin_memory()
                _build_from_host(W, host, sigma, 0).free()
                torch.cuda.synchronize()
                f0 = torch.cuda.Event(enable_timing=True)
                f1 = torch.cuda.Event(enable_timing=True)
                k2 = max(1, min(args.steps, 3))
                f0.record()
                for _ in range(k2):
                    _build_from_host(W, host, sigma, 0).free()
                f1.record()
                torch.cuda.synchronize()
                e2e = {"ms": reduce_max(f0.elapsed_time(f1) / k2, ws), "bytes": host.numel() * host.element_size()}
                del host
            del S
            torch.cuda.empty_cache()
    clk = clocks.stop()
    if rank != 0:
        return
    roofline, kernels, launches = roofline_of(stats, args.steps)
    line = {"metric": METRIC, "value": job_rate(n * len(per), ws, total_ms), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"locality stress (cont and rand): n={n} u32 codes, sigma=2^y for y in "
                                   f"{list(inputs.LOCALITY_SIZES)}; a step builds each of the {len(per)} inputs once",
                       "parallelism": f"replicas{ws}", "l2": "inputs (4 GiB each) larger than L2; no flush",
                       "inputs": per},
            "roofline": roofline, "cpu_baseline": None,
            "e2e": ({"value": job_rate(n, ws, e2e["ms"]), "unit": UNIT, "h2d_bytes_per_step": e2e["bytes"],
                     "d2h_bytes_per_step": 0, "input": f"rand, sigma=2^{inputs.LOCALITY_SIZES[-1]}"}
                    if e2e else None),
            "gpu_launches": launches, "clocks": clk, "kernels": kernels}
    print(json.dumps(line), flush=True)


MERGE_CHUNK_LOG2 = 28


def run_merge(args, ws, rank, local):
    """The buffered build of Section 5 on the default sequences: each of the
    text and DNA sequences (2^30 symbols) built in 2^28-symbol chunks, each
    chunk into a partial tree, then the partial trees merged into one
    (wt_build_chunked).  Reports the build rate, the merge step's own
    bandwidth, and the same build from pinned host buffers end to end."""
    import torch

    from paper_1610_05994_gb300 import build as B
    from paper_1610_05994_gb300 import wt as W

    torch.cuda.set_device(local)
    B.build_library()
    W.load()
    dev = torch.device("cuda", local)
    wls = WORKLOAD_SETS["text+dna"]
    host = [w.generate(min(w.n, 1 << args.size_log2) if args.size_log2 else None) for w in wls]
    sigmas = [w.sigma for w in wls]
    chunk = 1 << (min(MERGE_CHUNK_LOG2, args.size_log2 - 2) if args.size_log2 else MERGE_CHUNK_LOG2)
    seq_d = [torch.from_numpy(h).to(dev) for h in host]
    torch.cuda.synchronize()

    def step(src, keep):
        trees = [W.build_chunked(S, sigma, chunk, wait=False) for S, sigma in zip(src, sigmas)]
        for t in keep:
            t.free()
        return trees

    keep = []
    for _ in range(args.warmup):
        keep = step(seq_d, keep)
    for t in keep:
        t.wait()
    barrier(ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    W.profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        keep = step(seq_d, keep)
    e1.record()
    torch.cuda.synchronize()
    stats = W.profile_end()
    clk = clocks.stop()
    for t in keep:
        t.wait()
        t.free()
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, ws)
    syms = sum(h.size for h in host)

    host_p = [torch.from_numpy(h).pin_memory() for h in host]
    host_np = [p.numpy() for p in host_p]
    keep = step(host_np, [])
    for t in keep:
        t.wait()
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    k2 = max(1, min(args.steps, 3))
    f0.record()
    for _ in range(k2):
        keep = step(host_np, keep)
    f1.record()
    torch.cuda.synchronize()
    for t in keep:
        t.wait()
        t.free()
    ms_e2e = reduce_max(f0.elapsed_time(f1) / k2, ws)
    if rank != 0:
        return
    roofline, kernels, launches = roofline_of(stats, args.steps)
    mg = stats.get("merge")
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs") or 6800.0
    merge = None
    if mg and mg["total_ms"] > 0:
        gbs = mg["alg_bytes"] / (mg["total_ms"] * 1e-3) / 1e9
        merge = {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                 "alg_bytes_per_launch": mg["alg_bytes"] / mg["launches"],
                 "avg_launch_ms": mg["total_ms"] / mg["launches"],
                 "bytes_model": "per merged level of n bits: read the parts' bits n/8, write the level n/8 "
                                "and its directory n/128"}
    line = {"metric": METRIC, "value": job_rate(syms, ws, ms), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"buffered build (Section 5): u8 text n={host[0].size} sigma=96 Zipf(1.0) + "
                                   f"u8 DNA n={host[1].size} sigma=4 uniform, each in chunks of {chunk} symbols "
                                   f"built alone, then merged",
                       "chunk": chunk, "parallelism": f"replicas{ws}",
                       "l2": "inputs larger than L2; no flush"},
            "roofline": roofline, "merge_roofline": merge, "cpu_baseline": None,
            "e2e": {"value": job_rate(syms, ws, ms_e2e), "unit": UNIT,
                    "h2d_bytes_per_step": sum(h.nbytes for h in host), "d2h_bytes_per_step": 0,
                    "ms_per_step": ms_e2e},
            "gpu_launches": launches, "clocks": clk, "kernels": kernels}
    print(json.dumps(line), flush=True)


TUNE_CLASSES = [(4, 1, "uniform"), (20, 1, "zipf"), (96, 1, "zipf"), (256, 1, "uniform"), (1000, 2, "zipf"),
                 (65536, 2, "zipf"), (1 << 20, 4, "zipf")]
TUNE_LOG2N = (12, 14, 16, 18, 20, 22, 24, 26, 28)


def run_tune(args, ws, rank, local):
    """The autotuner's measurement: build time of every variant (one level
    per pass, two levels per pass, dd-direct where it applies) for each
    (alphabet, width) class and n = 2^12 .. 2^28, as the median device time
    between CUDA events around wt_build_async calls on the default stream
    (a small build is bound by its launches, so the host's launch cost is in
    the figure).  Prints one JSON line with the table and the fastest
    variant per entry."""
    import torch

    from paper_1610_05994_gb300 import build as B
    from paper_1610_05994_gb300 import wt as W

    torch.cuda.set_device(local)
    B.build_library()
    W.load()
    dev = torch.device("cuda", local)
    reps = max(3, args.steps)
    table = {}
    for sigma, width, dist in TUNE_CLASSES:
        dt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[width]
        big = (inputs.zipf(1 << max(TUNE_LOG2N), sigma, 1.0, 77, dt) if dist == "zipf"
               else inputs.uniform(1 << max(TUNE_LOG2N), sigma, 77, dt))
        big_d = torch.from_numpy(big).to(dev)
        row = {}
        for lg in TUNE_LOG2N:
            S = big_d[: 1 << lg]
            cells = {}
            variants = [W.VARIANT_LEVELWISE, W.VARIANT_PAIRS] + ([W.VARIANT_DD] if width == 1 else [])
            for var in variants:
                for _ in range(2):
                    W.Tree.build(S, sigma, variant=var).free()
                times = []
                for _ in range(reps):
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    torch.cuda.synchronize()
                    e0.record()
                    t = W.Tree.build(S, sigma, variant=var, wait=False)
                    e1.record()
                    t.wait()
                    times.append(e0.elapsed_time(e1))
                    t.free()
                cells[{1: "levelwise", 2: "dd", 3: "pairs"}[var]] = statistics.median(times)
            best = min(cells, key=cells.get)
            row[lg] = {"ms": cells, "best": best}
        table[f"sigma={sigma} w={width} {dist}"] = row
        del big_d
        torch.cuda.empty_cache()
    if rank != 0:
        return
    print(json.dumps({"metric": "build time per variant (ms, median)", "unit": "ms", "n_gpus": ws,
                      "reps": reps, "table": table}), flush=True)


def run_matrix(args, ws, rank, local):
    """Wavelet matrices of the default sequences (text and DNA, 2^30 symbols
    each): a step builds both, device-resident; the same builds from pinned
    host buffers end to end."""
    import ctypes as C

    import torch

    from paper_1610_05994_gb300 import build as B
    from paper_1610_05994_gb300 import wt as W

    torch.cuda.set_device(local)
    B.build_library()
    lib = W.load()
    dev = torch.device("cuda", local)
    wls = WORKLOAD_SETS["text+dna"]
    host = [w.generate(min(w.n, 1 << args.size_log2) if args.size_log2 else None) for w in wls]
    sigmas = [w.sigma for w in wls]
    seq_d = [torch.from_numpy(h).to(dev) for h in host]
    torch.cuda.synchronize()

    def step(keep):
        trees = [W.Tree.build(S, sigma, wait=False, matrix=True) for S, sigma in zip(seq_d, sigmas)]
        for t in keep:
            t.free()
        return trees

    keep = []
    for _ in range(args.warmup):
        keep = step(keep)
    for t in keep:
        t.wait()
    barrier(ws)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    W.profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        keep = step(keep)
    e1.record()
    torch.cuda.synchronize()
    stats = W.profile_end()
    clk = clocks.stop()
    for t in keep:
        t.wait()
        t.free()
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, ws)
    syms = sum(h.size for h in host)

    host_p = [torch.from_numpy(h).pin_memory() for h in host]

    def step_host(keep):
        trees = []
        for p, sigma in zip(host_p, sigmas):
            h = lib.wt_build_matrix_async(C.c_void_p(p.data_ptr()), p.numel(), sigma, p.element_size(),
                                          C.c_void_p(W._stream(None)))
            if not h:
                raise W.WTError(lib.wt_last_status(), "wt_build_matrix_async")
            trees.append(W.Tree(h, p.numel(), sigma, p.element_size()))
        for t in keep:
            t.free()
        return trees

    keep = step_host([])
    torch.cuda.synchronize()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    k2 = max(1, min(args.steps, 3))
    f0.record()
    for _ in range(k2):
        keep = step_host(keep)
    f1.record()
    torch.cuda.synchronize()
    for t in keep:
        t.wait()
        t.free()
    ms_e2e = reduce_max(f0.elapsed_time(f1) / k2, ws)
    if rank != 0:
        return
    roofline, kernels, launches = roofline_of(stats, args.steps)
    line = {"metric": "wavelet-matrix build symbols/sec", "value": job_rate(syms, ws, ms), "unit": UNIT,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": f"wavelet matrices (Section 5, Claude and Navarro 2012): u8 text n={host[0].size} "
                                   f"sigma=96 Zipf(1.0) + u8 DNA n={host[1].size} sigma=4 uniform, builds only",
                       "parallelism": f"replicas{ws}", "l2": "inputs larger than L2; no flush"},
            "roofline": roofline, "cpu_baseline": None,
            "e2e": {"value": job_rate(syms, ws, ms_e2e), "unit": UNIT,
                    "h2d_bytes_per_step": sum(h.nbytes for h in host), "d2h_bytes_per_step": 0,
                    "ms_per_step": ms_e2e},
            "gpu_launches": launches, "clocks": clk, "kernels": kernels}
    print(json.dumps(line), flush=True)


def roofline_of(stats: dict, steps: int):
    """Roofline of the kernel with the largest device time, per-kernel
    figures per step, and the number of library launches, from the library's
    own launch profile (CUDA events on the launching stream)."""
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peak else "fallback (6800 GB/s)"
    peak = peak or 6800.0
    roofline = None
    if stats:
        name, st = max(stats.items(), key=lambda kv: kv[1]["total_ms"])
        achieved = st["alg_bytes"] / (st["total_ms"] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": peak_src, "traffic": ncu_traffic(name),
                    "alg_bytes_per_launch": st["alg_bytes"] / st["launches"],
                    "avg_launch_ms": st["total_ms"] / st["launches"]}
        if st.get("variant_bytes"):
            vb = st["variant_bytes"] / (st["total_ms"] * 1e-3) / 1e9
            roofline["variant_bytes_achieved"] = vb
            roofline["variant_bytes_frac"] = vb / peak
        # The whole build against the level-wise model's total bytes (the
        # histogram term n w is the read of S for the counts: the histogram,
        # or level 0's count pass when the node tables come by rank).
        build = [k for k in ("histogram", "level0_count", "node_starts", "node_tables", "level_pass") if k in stats]
        if "level_pass" in build:
            b_bytes = sum(stats[k]["alg_bytes"] for k in build if k in ("histogram", "level0_count", "level_pass"))
            b_ms = sum(stats[k]["total_ms"] for k in build)
            ach = b_bytes / (b_ms * 1e-3) / 1e9
            roofline["build"] = {"kernels": build, "achieved": ach, "frac": ach / peak,
                                 "ms_per_step": b_ms / steps}
    kernels = {k: {"launches": v["launches"], "cuda_kernels": v["kernels"], "ms_per_step": v["total_ms"] / steps,
                   "GBps": v["alg_bytes"] / (v["total_ms"] * 1e-3) / 1e9 if v["total_ms"] > 0 else None}
               for k, v in stats.items()}
    return roofline, kernels, sum(v["kernels"] for v in stats.values())


def _gen_parallel(specs):
    """Host sequences of many specs, generated on all host cores."""
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(min(32, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda sp: sp.generate(), specs))


def _pack_device(host, dev, align=256):
    """Copies host sequences into one device buffer (each start aligned) and
    returns typed views of it, one per sequence."""
    import torch
    offs, total = [], 0
    for h in host:
        offs.append(total)
        total += (h.nbytes + align - 1) // align * align
    stage = torch.empty(max(total, 1), dtype=torch.uint8).pin_memory()
    sv = stage.numpy()
    for h, o in zip(host, offs):
        sv[o:o + h.nbytes] = h.view(np.uint8)
    buf = stage.to(dev)
    tdt = {1: torch.uint8, 2: torch.uint16, 4: torch.int32}
    return buf, [buf[o:o + h.nbytes].view(tdt[h.itemsize]) for h, o in zip(host, offs)]


BATCH_CLASS_N = 1 << 28


def run_batch(args, ws, rank, local):
    """Batched build of 4096 sequences per step (one wt_build_batch call, one
    CUDA graph), and the plain path's rate on one 2^28-symbol sequence of each
    (alphabet, distribution) class, for the efficiency figure."""
    import torch

    from paper_1610_05994_gb300 import build as B
    from paper_1610_05994_gb300 import wt as W

    torch.cuda.set_device(local)
    B.build_library()
    W.load()
    dev = torch.device("cuda", local)
    specs = inputs.batch_specs(args.batch_count, base=inputs.SEED_BASE + 4 + 1000 * rank)
    t_gen = time.perf_counter()
    host = _gen_parallel(specs)
    t_gen = time.perf_counter() - t_gen
    buf, seqs = _pack_device(host, dev)
    sigmas = [sp.sigma for sp in specs]
    n_total = sum(sp.n for sp in specs)
    st = torch.cuda.Stream(dev)
    torch.cuda.synchronize()

    host_ms = []  # host time of each wt_build_batch call (plan, uploads, graph capture and launch)

    def step(keep):
        h0 = time.perf_counter()
        trees = W.build_batch(seqs, sigmas, stream=st, wait=False)
        host_ms.append((time.perf_counter() - h0) * 1e3)
        with torch.cuda.stream(st):
            for t in keep:
                t.free()
        return trees

    keep = []
    for _ in range(args.warmup):
        keep = step(keep)
    for t in keep:
        t.wait()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    W.profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(ws)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        keep = step(keep)
    e1.record(st)
    torch.cuda.synchronize()
    barrier(ws)
    stats = W.profile_end()
    clk = clocks.stop()
    for t in keep:
        t.wait()
        t.free()
    ms = reduce_max(e0.elapsed_time(e1) / args.steps, ws)
    value = job_rate(n_total, ws, ms)

    # End to end: inputs copied from pinned host memory inside the timed region.
    stage = torch.empty(buf.numel(), dtype=torch.uint8).pin_memory()
    stage.copy_(buf)
    keep = []
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    f0.record(st)
    e2e_steps = max(1, min(args.steps, 3))
    for _ in range(e2e_steps):
        with torch.cuda.stream(st):
            buf.copy_(stage, non_blocking=True)
        keep = step(keep)
    f1.record(st)
    torch.cuda.synchronize()
    for t in keep:
        t.wait()
        t.free()
    ms_e2e = reduce_max(f0.elapsed_time(f1) / e2e_steps, ws)
    del buf, seqs, stage

    # Plain path per class: sigma x distribution, one 2^28-symbol sequence each.
    classes = sorted({(sp.sigma, sp.width, sp.dist) for sp in specs})
    rate = {}
    for k, (sigma, width, dist) in enumerate(classes):
        sp = inputs.SeqSpec(BATCH_CLASS_N, sigma, width, dist, 1.1 if dist == "zipf" else 0.0,
                            inputs.seq_seed(inputs.SEED_BASE + 40, k))
        S = torch.from_numpy(sp.generate()).to(dev)
        for _ in range(2):
            W.Tree.build(S, sigma).free()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        reps = 3
        c0.record()
        for _ in range(reps):
            W.Tree.build(S, sigma, wait=False).free()
        c1.record()
        torch.cuda.synchronize()
        rate[(sigma, width, dist)] = BATCH_CLASS_N / (c0.elapsed_time(c1) / reps * 1e-3)
        del S
    plain_sec = sum(sp.n / rate[(sp.sigma, sp.width, sp.dist)] for sp in specs)
    efficiency = plain_sec / (ms * 1e-3)
    if rank != 0:
        return
    roofline, kernels, launches = roofline_of(stats, args.steps)
    h2d = sum(h.nbytes for h in host)
    line = {"metric": "batched wavelet-tree build symbols/sec", "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8+u16", "data": "synthetic",
            "config": {"workload": f"batch of {args.batch_count} sequences, n log-uniform in [2^10, 2^22], sigma in "
                                   "{4, 20, 256, 65536} (u8 for sigma <= 256, else u16), uniform or Zipf(1.1)",
                       "symbols_per_step": n_total, "host_generation_s": t_gen,
                       "l2": "inputs (2.6 GB) larger than the 129 MB L2; no flush",
                       "parallelism": f"replicas{ws}"},
            "batch_efficiency_vs_plain": efficiency,
            "host_ms_per_call": float(np.median(host_ms[args.warmup:] or host_ms)),
            "plain_rate_per_class": {f"sigma={k[0]} w={k[1]} {k[2]}": v for k, v in rate.items()},
            "roofline": roofline, "cpu_baseline": None,
            "e2e": {"value": job_rate(n_total, ws, ms_e2e), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": 0, "ms_per_step": ms_e2e},
            "gpu_launches": launches, "clocks": clk, "kernels": kernels}
    print(json.dumps(line), flush=True)


SERVE_POOL_N = 1 << 26


def _serve_phase(srv, BuildRequest, specs, offs, pools, hists, lam, warm, rng, qrng, arrive):
    """Runs one serving phase: Poisson arrivals at rate lam, the server's
    steps, and closed-loop query batches on the resident trees.  Returns the
    measured requests (rid >= warm), the measured query batches and the
    phase's wall time."""
    import torch

    total = len(specs)
    arrivals = np.cumsum(rng.exponential(1.0 / lam, total))
    where = {}  # rid -> (sigma, offset, n)
    qbs = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    k = 0
    qb = None
    while len(srv.finished) + len(srv.failed) + len(srv.rejected) < total:
        now = time.perf_counter() - t0
        while k < total and arrivals[k] <= now:
            where[k] = (specs[k].sigma, offs[k], specs[k].n)
            srv.submit(BuildRequest(k, arrive(k), specs[k].sigma, t0 + arrivals[k]))
            k += 1
        srv.step()
        srv.poll_queries()
        if srv.resident and (qb is None or qb.done):
            rids = list(srv.resident)
            tidx, op, c, arg = _serve_queries(qrng, rids, where, pools, hists, QUERIES)
            q = [torch.from_numpy(x).to(srv.device, non_blocking=False) for x in (tidx, op, c, arg)]
            qb = srv.query([srv.resident[r][0] for r in rids], *q)
            qb.measured = k > warm
            qbs.append(qb)
    srv.drain()
    meas = [r for r in srv.finished if r.rid >= warm]
    q_meas = [q for q in qbs if getattr(q, "measured", False) and q.done]
    return meas, q_meas, time.perf_counter() - t0


def run_serve(args, ws, rank, local):
    """Serving loop: Poisson arrivals of build requests at an offered load of
    70% of the measured batched build rate, continuous batching under a 120 GB
    budget, closed-loop batches of 2^16 mixed queries on the resident trees.
    A second phase offers requests until the resident trees reach the budget,
    so that admission evicts the oldest trees."""
    import torch

    from paper_1610_05994_gb300 import build as B
    from paper_1610_05994_gb300 import wt as W
    from paper_1610_05994_gb300.serve import BuildRequest, Server, percentiles, resident_bytes

    torch.cuda.set_device(local)
    B.build_library()
    W.load()
    dev = torch.device("cuda", local)
    budget = 120 << 30
    warm, total = 100, 100 + args.requests
    specs = inputs.serving_specs(total, base=inputs.SEED_BASE + 5 + 1000 * rank)
    # Request data: slices of one pinned Zipf(1.0) pool per alphabet, at
    # seeded offsets; each request is copied to the device when it arrives.
    pools, hists = {}, {}
    for k, sigma in enumerate((256, 65536)):
        h = inputs.zipf(SERVE_POOL_N, sigma, 1.0, inputs.seq_seed(inputs.SEED_BASE + 50, k))
        pools[sigma] = torch.from_numpy(h).pin_memory()
        hists[sigma] = np.bincount(h, minlength=sigma).astype(np.float64) / SERVE_POOL_N
    rng = np.random.default_rng(55 + rank)
    offs = [int(rng.integers(0, SERVE_POOL_N - sp.n + 1)) for sp in specs]

    def arriver(sp_list, off_list):
        def arrive(k):
            sp = sp_list[k]
            S = torch.empty(sp.n, dtype=pools[sp.sigma].dtype, device=dev)
            S.copy_(pools[sp.sigma][off_list[k]:off_list[k] + sp.n], non_blocking=True)
            return S
        return arrive

    arrive = arriver(specs, offs)
    # Calibration on 64 requests of this distribution: the batched build
    # rate (one wt_build_batch call) and the plain rate (each request built
    # alone, one after the other).
    cal = [arrive(k) for k in range(64)]
    cal_sig = [specs[k].sigma for k in range(64)]
    cal_n = sum(specs[k].n for k in range(64))
    for _ in range(2):
        for t in W.build_batch(cal, cal_sig):
            t.free()
        for S, sg in zip(cal, cal_sig):
            W.Tree.build(S, sg).free()
    torch.cuda.synchronize()
    c0 = time.perf_counter()
    for t in W.build_batch(cal, cal_sig):
        t.free()
    torch.cuda.synchronize()
    batch_rate = cal_n / (time.perf_counter() - c0)
    c0 = time.perf_counter()
    for S, sg in zip(cal, cal_sig):
        W.Tree.build(S, sg, wait=False).free()
    torch.cuda.synchronize()
    plain_rate = cal_n / (time.perf_counter() - c0)
    del cal
    mean_n = float(np.mean([sp.n for sp in specs]))
    lam = 0.7 * batch_rate / mean_n

    # Phase 1: the measured serving run.
    srv = Server(budget_bytes=budget, max_batch=1024, device=dev)
    qrng = np.random.default_rng(77 + rank)
    clocks = ClockSampler(local)
    clocks.start()
    W.profile_begin()
    meas, qbs, wall = _serve_phase(srv, BuildRequest, specs, offs, pools, hists, lam, warm, rng, qrng, arrive)
    stats = W.profile_end()
    clk = clocks.stop()
    first = min(r.arrival for r in meas)
    last = max(r.done for r in meas)
    # replicas: every rank serves its own stream; the job's rate is all the
    # symbols served over the slowest rank's span
    span_s = reduce_max(last - first, ws)
    value = reduce_sum(sum(r.n for r in meas), ws) / span_s
    build_lat = [(r.done - r.arrival) * 1e3 for r in meas]
    wait_lat = [(r.admitted - r.arrival) * 1e3 for r in meas]
    q_lat = [(q.done - q.issued) * 1e3 for q in qbs]
    phase1 = {"evicted": srv.evicted, "peak_used_gb": srv.peak_used / 2**30, "build_batches": srv.batches,
              "batch_host_ms": percentiles(srv.batch_host_ms), "rejected": len(srv.rejected),
              "failed": len(srv.failed)}
    srv.close()

    # Phase 2, at the budget: enough requests that the resident trees fill
    # the 120 GB and admission evicts the oldest ones.
    mean_keep = float(np.mean([resident_bytes(sp.n, sp.sigma) for sp in specs]))
    total2 = int(1.3 * budget / mean_keep) + warm
    specs2 = inputs.serving_specs(total2, base=inputs.SEED_BASE + 6 + 1000 * rank)
    offs2 = [int(rng.integers(0, SERVE_POOL_N - sp.n + 1)) for sp in specs2]
    srv2 = Server(budget_bytes=budget, max_batch=1024, device=dev)
    meas2, qbs2, wall2 = _serve_phase(srv2, BuildRequest, specs2, offs2, pools, hists, lam, warm, rng, qrng,
                                      arriver(specs2, offs2))
    first2 = min(r.arrival for r in meas2)
    last2 = max(r.done for r in meas2)
    at_cap = {"requests": total2 - warm, "value": sum(r.n for r in meas2) / (last2 - first2), "unit": UNIT,
              "evicted": srv2.evicted, "peak_used_gb": srv2.peak_used / 2**30, "budget_gb": budget / 2**30,
              "rejected": len(srv2.rejected), "failed": len(srv2.failed), "build_batches": srv2.batches,
              "latency_ms": {"build": percentiles([(r.done - r.arrival) * 1e3 for r in meas2]),
                             "admission_wait": percentiles([(r.admitted - r.arrival) * 1e3 for r in meas2]),
                             "query_batch": percentiles([(q.done - q.issued) * 1e3 for q in qbs2])},
              "batch_host_ms": percentiles(srv2.batch_host_ms), "wall_s": wall2}
    srv2.close()
    if rank != 0:
        return
    roofline, kernels, launches = roofline_of(stats, 1)
    line = {"metric": "served wavelet-tree build symbols/sec", "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.requests, "warmup": warm, "ms_per_step": (last - first) * 1e3 / len(meas),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8+u16",
            "data": "synthetic",
            "config": {"workload": "serving: Poisson build requests, n log-uniform in [2^12, 2^26], sigma in "
                                   "{256 (u8), 65536 (u16)}, Zipf(1.0); closed-loop batches of 2^16 mixed "
                                   "access/rank/select queries on resident trees; 120 GB admission budget",
                       "requests": args.requests, "warmup_requests": warm, "offered_load": 0.7,
                       "calibrated_batch_rate": batch_rate, "calibrated_plain_rate": plain_rate,
                       "arrival_rate_per_s": lam, "parallelism": f"replicas{ws}"},
            "served_vs_batch_rate": value / batch_rate, "served_vs_plain_rate": value / plain_rate,
            "batch_vs_plain_rate": batch_rate / plain_rate,
            "latency_ms": {"build": percentiles(build_lat), "admission_wait": percentiles(wait_lat),
                           "query_batch": percentiles(q_lat)},
            "queries_per_s": QUERIES * len(q_lat) / (last - first) if q_lat else None,
            "query_batches": len(q_lat), **phase1, "at_capacity": at_cap,
            "wall_s": wall, "roofline": roofline, "cpu_baseline": None,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": float(np.mean(
                        [specs[r.rid].n * specs[r.rid].width for r in meas])), "d2h_bytes_per_step": 0,
                    "note": "the value itself is end to end: request data is copied from pinned host "
                            "memory after arrival, inside each request's latency"},
            "gpu_launches": launches, "clocks": clk, "kernels": kernels}
    print(json.dumps(line), flush=True)


def _serve_queries(rng, rids, where, pools, hists, m):
    """A batch of m mixed queries over the resident trees: uniform tree, op
    and position; c drawn from the tree's sequence; j within the symbol's
    expected count."""
    tidx = rng.integers(0, len(rids), m).astype(np.uint32)
    op = rng.integers(0, 3, m).astype(np.uint8)
    sig = np.array([where[r][0] for r in rids], np.int64)[tidx]
    off = np.array([where[r][1] for r in rids], np.int64)[tidx]
    n = np.array([where[r][2] for r in rids], np.int64)[tidx]
    pos = (rng.random(m) * n).astype(np.int64)
    c = np.zeros(m, np.uint32)
    cnt = np.zeros(m, np.float64)
    for sigma, pool in pools.items():
        sel = sig == sigma
        c[sel] = pool.numpy()[off[sel] + pos[sel]]
        cnt[sel] = hists[sigma][c[sel]] * n[sel]
    i_arg = (rng.random(m) * (n + 1)).astype(np.uint64)
    j_arg = (1 + np.floor(rng.random(m) * np.maximum(np.floor(cnt), 1))).astype(np.uint64)
    arg = np.where(op == 2, j_arg, i_arg).astype(np.uint64)
    return tidx, op, c, arg


def _build_from_host(W, pinned, sigma, variant):
    """wt_build_async from a pinned host buffer (the library stages the copy)."""
    import ctypes as C
    lib = W.load()
    h = lib.wt_build_async(C.c_void_p(pinned.data_ptr()), pinned.numel(), sigma, pinned.element_size(),
                           variant, C.c_void_p(W._stream(None)))
    if not h:
        raise W.WTError(lib.wt_last_status(), "wt_build_async")
    return W.Tree(h, pinned.numel(), sigma, pinned.element_size())


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    runners = {"batch": run_batch, "serve": run_serve, "locality": run_locality, "merge": run_merge, "tune": run_tune,
               "matrix": run_matrix}
    ap.add_argument("--workload", choices=sorted(WORKLOAD_SETS) + sorted(runners), default="text+dna")
    ap.add_argument("--requests", type=int, default=2000, help="serve: measured build requests")
    ap.add_argument("--batch-count", type=int, default=4096,
                    help="batch: sequences per step (profiling aid; the line then names the count)")
    ap.add_argument("--size-log2", type=int, default=0,
                    help="profiling aid: cap each sequence at 2^k symbols (the line then names the cap)")
    ap.add_argument("--variant", type=int, choices=[0, 1, 2, 3], default=0,
                    help="0 auto (autotuned), 1 level-wise, 2 dd-direct, 3 two levels per pass")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        if args.workload in runners:
            print(json.dumps({"impl": "reference", "unavailable": "the oracle is timed on the single-sequence "
                              "workloads only"}), flush=True)
            return
        run_reference(args, ws, rank)
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        RUN.update(workload=args.workload, size_log2=args.size_log2, variant=args.variant)
        runners.get(args.workload, run_ours)(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
