#!/usr/bin/env python3
"""Throughput bench of the GB300 Toeplitz hash (privacy amplification, arXiv 1805.02372).

One step = one pass of the whole hot path over the workload's blocks: plan lookup,
the decomposition into tiles, the kernels, the XOR merge, packed output. Inputs are
seeded synthetic uniform bits, resident in HBM before the timed region; the metric
is input-key Gbps (sum of n over the blocks / device time, Mbit = 10^6 bits as in
Table 1), bit-exact against the CPU oracle (checked on sampled rows every run).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                       [--path auto|direct|ntt64|ntt31|fft|block_int8] [--impl ours|reference]
Under torchrun every rank runs the same workload on its own GPU (independent
blocks: weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
METRIC = "input-key Gbps per GB300 (bit-exact) batched vs plain kernel; p99 latency"
UNIT = "Gbps"


# --------------------------------------------------------------------------- workloads

def workload(name: str):
    from paper_1805_02372_gb300 import inputs
    if name == "batched256":
        return inputs.batched_blocks(), {
            "workload": "batched: 256 independent blocks, n_i log-uniform in [1e5, 4e6], "
                        "r_i uniform in [0.01, 0.5], m_i = floor(r_i n_i), fresh seed per block",
            "blocks": 256}
    if name == "plain_single":
        b = inputs.PLAIN_SINGLE
        return [b], {"workload": f"plain single block n={b.n} m={b.m}", "blocks": 1}
    if name.startswith("plain_vs_transform"):
        m = int(name.split("_m")[-1]) if "_m" in name else 500_000
        b = inputs.single_block(1_000_000, m)
        return [b], {"workload": f"plain vs transform n={b.n} m={b.m}", "blocks": 1}
    if name == "finite_size":
        b = inputs.FINITE_SIZE
        return [b], {"workload": f"finite-size scale n={b.n} m={b.m}", "blocks": 1}
    raise SystemExit(f"unknown workload {name}")


# --------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return None
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------- runners

class Runner:
    """Device-resident buffers + plans for a list of blocks; one step = all blocks."""

    def __init__(self, blocks, path: str, device):
        import torch

        import paper_1805_02372_gb300 as pkg
        self.pkg, self.torch = pkg, torch
        self.blocks = blocks
        self.path = path
        self.keys_h = [b.key() for b in blocks]
        self.seeds_h = [b.seed() for b in blocks]
        t = lambda a: torch.from_numpy(a.view(np.int64)).to(device)
        self.keys = [t(k) for k in self.keys_h]
        self.seeds = [t(s) for s in self.seeds_h]
        self.outs = [torch.zeros((b.m + 63) // 64, dtype=torch.int64, device=device)
                     for b in blocks]
        self.batched = len(blocks) > 1
        self.stream = torch.cuda.current_stream()
        if self.batched:
            self.desc = [(b.n, b.m, s, k, o) for b, s, k, o in
                         zip(blocks, self.seeds, self.keys, self.outs)]
            self.batch = pkg.pa_batch_plan(self.desc, pkg.make_opts(path=path))
            self.plans = None
        else:
            self.plans = [pkg.Plan(b.n, b.m, path=path) for b in blocks]
        self.units = sum(b.n for b in blocks)

    def step(self):
        if self.batched:
            self.pkg.pa_batch_run(self.batch, self.desc, self.stream)
        else:
            for p, s, k, o in zip(self.plans, self.seeds, self.keys, self.outs):
                p.hash(s, k, o, self.stream)

    def profile(self, on: bool):
        if self.batched:
            self.pkg.pa_batch_profile(self.batch, on)
        else:
            for p in self.plans:
                self.pkg.pa_plan_profile(p.handle, on)

    def kernel_times(self) -> dict:
        if self.batched:
            return self.pkg.pa_batch_kernel_times(self.batch)
        tot = {}
        for p in self.plans:
            for k, v in self.pkg.pa_plan_kernel_times(p.handle).items():
                t = tot.setdefault(k, {"launches": 0, "total_ms": 0.0})
                t["launches"] += v["launches"]
                t["total_ms"] += v["total_ms"]
        return tot

    def describe(self):
        if self.batched:
            rep = self.pkg.pa_batch_run(self.batch, self.desc, self.stream, report=True)
            return {"report": rep}
        return {"plans": [p.desc for p in self.plans]}


def check_sampled(runner, rows_per_block=64, seed=7):
    """Bit-exact check of the last step's outputs on sampled rows (oracle, CPU)."""
    import oracle
    rng = np.random.default_rng(seed)
    bad = 0
    for b, k, s, o in zip(runner.blocks, runner.keys_h, runner.seeds_h, runner.outs):
        rows = np.unique(np.concatenate([[0, b.m - 1], rng.integers(0, b.m, rows_per_block)]))
        want = oracle.hash_rows(b.n, b.m, s, k, rows)
        got = oracle.unpack(o.cpu().numpy().view(np.uint64), b.m)[rows]
        bad += int((want != got).sum())
    return bad == 0


# --------------------------------------------------------------------------- roofline

def _source_digest(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {
    "direct": ["paper_1805_02372_gb300/csrc/direct.cu", "paper_1805_02372_gb300/csrc/common.cuh"],
}


def algorithmic(kernel: str, blocks, launches_per_step: int):
    """(bound, algorithmic units per launch, unit). Counts per DESIGN's roofline section."""
    if kernel == "direct":
        # 32 funnel shifts + 32 LOP3 per 32 rows x 32 key bits: m*n/16 integer ops.
        ops = sum(2.0 * b.m * b.n / 32.0 for b in blocks) / launches_per_step
        return "alu", ops, "Tops/s"
    return None, None, None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def roofline(kt: dict, blocks, steps: int, clocks):
    if not kt:
        return None
    dom = max(kt.items(), key=lambda kv: kv[1]["total_ms"])
    name, v = dom
    per_launch_ms = v["total_ms"] / max(v["launches"], 1)
    launches_per_step = max(1, round(v["launches"] / steps))
    bound, units, unit = algorithmic(name, blocks, launches_per_step)
    pk, src = peaks()
    out = {"kernel": name, "launch_ms": per_launch_ms, "launches": v["launches"]}
    if bound == "alu":
        # 152 SMs x 64 INT32 (LOP3/SHF) lanes x max SM clock (2070 MHz).
        peak = 152 * 64 * 2070e6 / 1e12
        ach = units / (per_launch_ms * 1e-3) / 1e12
        out.update({"bound": "alu", "achieved": ach, "peak": peak, "unit": unit,
                    "frac": ach / peak, "peak_source": "derived: 152 SM x 64 INT32 lanes x 2070 MHz"})
    elif bound == "hbm":
        peak = pk["hbm_gbs"]
        ach = units / (per_launch_ms * 1e-3) / 1e9
        out.update({"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                    "frac": ach / peak, "peak_source": src})
    out["traffic"] = traffic_for(name)
    out["share"] = v["total_ms"] / sum(x["total_ms"] for x in kt.values())
    return out


def traffic_for(kernel: str):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            tab = json.load(f)
    except (OSError, ValueError):
        return None
    ent = tab.get(kernel)
    if not ent or kernel not in KERNEL_SOURCES:
        return None
    if ent.get("source_digest") != _source_digest(KERNEL_SOURCES[kernel]):
        return None
    return ent.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- CPU oracle

def cpu_oracle_gbps(blocks, budget_s: float = 12.0, seed: int = 3):
    """The oracle as it stands on a bounded uniform sample of output rows of the workload.

    Rows are drawn uniformly over all sum(m) rows; the full-job time is the sample time
    scaled by sum(m) / rows. Returns (Gbps, cores, description)."""
    import oracle
    rng = np.random.default_rng(seed)
    total_m = sum(b.m for b in blocks)
    avg_n = sum(b.n * b.m for b in blocks) / total_m
    # calibrate: oracle row cost ~ n/64 word ops; start small, grow to the budget
    rows_total = max(8, int(2000 * 1e6 / avg_n))
    spent, done_rows, elapsed = 0.0, 0, 0.0
    keys = {}
    while spent < budget_s:
        pick = rng.integers(0, total_m, rows_total)
        edges = np.cumsum([0] + [b.m for b in blocks])
        which = np.searchsorted(edges, pick, side="right") - 1
        t0 = time.perf_counter()
        for bi in np.unique(which):
            b = blocks[bi]
            if bi not in keys:
                keys[bi] = (b.key(), b.seed())
            k, s = keys[bi]
            rows = pick[which == bi] - edges[bi]
            oracle.hash_rows(b.n, b.m, s, k, rows)
        dt = time.perf_counter() - t0
        spent += dt
        elapsed += dt
        done_rows += rows_total
        if dt < budget_s / 8:
            rows_total *= 4
    full_s = elapsed * total_m / done_rows
    gbps = sum(b.n for b in blocks) / full_s / 1e9
    cores = os.cpu_count() or 1
    return gbps, cores, (f"{done_rows} output rows drawn uniformly from the workload's "
                         f"{total_m} rows ({elapsed:.1f} s), scaled by sum(m)/rows")


# --------------------------------------------------------------------------- main

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    blocks, cfg = workload(args.workload)
    per_step = []
    for _ in range(args.warmup):
        cpu_oracle_gbps(blocks, budget_s=2.0)
    for k in range(args.steps):
        g, cores, desc = cpu_oracle_gbps(blocks, budget_s=8.0, seed=100 + k)
        per_step.append(g)
    val = float(np.mean(per_step))
    total_bits = sum(b.n for b in blocks)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_bits / (val * 1e9) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": cfg,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="plain_vs_transform_m500000")
    ap.add_argument("--path", default="auto")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=device)

    blocks, cfg = workload(args.workload)
    runner = Runner(blocks, args.path, device)
    stream = runner.stream
    for _ in range(args.warmup):
        runner.step()
    torch.cuda.synchronize()

    in_bytes = sum(8 * (len(k) + len(s)) for k, s in zip(runner.keys_h, runner.seeds_h))
    flush = in_bytes < 2 * L2_BYTES
    scratch = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=device) if flush else None
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    runner.profile(True)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for a, b in evs:
            if flush:
                scratch.add_(1)
            a.record(stream)
            runner.step()
            b.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    runner.profile(False)
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    if world > 1:
        t = torch.tensor([ms], device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
        dist.barrier()
    kt = runner.kernel_times()
    exact = check_sampled(runner)
    clocks = clk.summary()

    # e2e through the public host-buffer entry point, copies inside the timed region
    e2e = None
    if not runner.batched:
        p = runner.plans[0]
        b = blocks[0]
        kh = torch.from_numpy(runner.keys_h[0].view(np.int64)).pin_memory()
        sh = torch.from_numpy(runner.seeds_h[0].view(np.int64)).pin_memory()
        oh = torch.zeros((b.m + 63) // 64, dtype=torch.int64).pin_memory()
        p.hash_host(sh, kh, oh, stream)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            p.hash_host(sh, kh, oh, stream)
        dt = (time.perf_counter() - t0) / args.steps
        e2e = {"value": b.n / dt / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": int(kh.numel() * 8 + sh.numel() * 8),
               "d2h_bytes_per_step": int(oh.numel() * 8)}

    units = runner.units * world
    value = units / (ms * 1e-3) / 1e9
    launches = sum(v["launches"] for k, v in kt.items() if k != "memset") // args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": dict(cfg, path=args.path, l2="flushed between steps" if flush else
                       "inputs larger than L2", bit_exact_sampled=exact),
        "roofline": roofline(kt, blocks, args.steps, clocks),
        "e2e": e2e, "gpu_launches": launches * args.steps, "clocks": clocks,
        "kernel_times_ms": {k: round(v["total_ms"] / args.steps, 5) for k, v in kt.items()},
        "wall_s": wall,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, cores, desc = cpu_oracle_gbps(blocks)
        line["cpu_baseline"] = {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
