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
ORACLE_SAMPLE = {"text+dna": 1 << 27, "words": 1 << 24}     # cpu_baseline: 10-30 s of oracle work
REFERENCE_SAMPLE = {"text+dna": 1 << 26, "words": 1 << 23}  # --impl reference, per step


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


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


def source_hash() -> str:
    h = hashlib.sha256()
    for f in sorted(os.listdir(os.path.join(ROOT, "paper_1610_05994_gb300", "csrc"))):
        with open(os.path.join(ROOT, "paper_1610_05994_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was taken on the current kernel sources; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("source_hash") != source_hash():
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
    host = [w.generate() for w in wls]
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

    def barrier():
        if ws > 1:
            dist.barrier()

    keep = []
    for _ in range(args.warmup):
        keep = step(keep)
    for t in keep:
        t.wait()
    barrier()
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    W.profile_begin()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.steps):
        keep = step(keep)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    stats = W.profile_end()
    clk = clocks.stop()
    for t in keep:
        t.wait()
        t.free()
    keep = []
    ms = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        tt = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    syms_rank = sum(w.n for w in wls)
    syms = syms_rank * ws
    value = syms / (ms * 1e-3)

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
    barrier()
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
    ms_e2e = f0.elapsed_time(f1) / e2e_steps
    if ws > 1:
        tt = torch.tensor([ms_e2e], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_e2e = float(tt.item())
    h2d = sum(h.nbytes for h in host) + sum(x.numel() * x.element_size() for x in q_p)
    d2h = QUERIES * 8

    if rank != 0:
        return
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peak else "fallback (6800 GB/s)"
    peak = peak or 6800.0
    dom = max(stats.items(), key=lambda kv: kv[1]["total_ms"]) if stats else (None, None)
    roofline = None
    if dom[0]:
        name, st = dom
        achieved = st["alg_bytes"] / (st["total_ms"] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                    "frac": achieved / peak, "peak_source": peak_src, "traffic": ncu_traffic(name),
                    "alg_bytes_per_launch": st["alg_bytes"] / st["launches"],
                    "avg_launch_ms": st["total_ms"] / st["launches"]}
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["total_ms"] / args.steps,
                   "GBps": v["alg_bytes"] / (v["total_ms"] * 1e-3) / 1e9 if v["total_ms"] > 0 else None}
               for k, v in stats.items()}
    launches = sum(v["launches"] for v in stats.values())
    cpu = None if args.no_cpu_baseline or ws > 1 else cpu_baseline_sample(args.workload)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype_of(args.workload), "data": "synthetic",
            "config": dict(config_for(args.workload), parallelism=f"replicas{ws}",
                           variant={0: "auto", 1: "levelwise", 2: "dd"}[args.variant]),
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": syms / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": ms_e2e},
            "gpu_launches": launches, "clocks": clk, "kernels": kernels}
    print(json.dumps(line), flush=True)


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
    ap.add_argument("--workload", choices=sorted(WORKLOAD_SETS), default="text+dna")
    ap.add_argument("--variant", type=int, choices=[0, 1, 2], default=0,
                    help="0 auto (autotuned), 1 level-wise, 2 dd-direct")
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
