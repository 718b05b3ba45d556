#!/usr/bin/env python3
"""Throughput bench of the GB300 Toeplitz hash (privacy amplification, arXiv 1805.02372).

One step = one pass of the whole hot path over the workload's blocks: plan lookup,
the decomposition into tiles, the kernels, the XOR merge, packed output. Inputs are
seeded synthetic uniform bits, resident in HBM before the timed region; the metric
is input-key Gbps (sum of n over the blocks / device time, Mbit = 10^6 bits as in
Table 1), bit-exact against the CPU oracle (checked on sampled rows every run).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                       [--path auto|direct|ntt64|ntt31|fft|block_int8|block_fp8]
                       [--impl ours|reference]
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
    if name.startswith("batched") and name != "batched256":
        k = int(name[len("batched"):])
        return inputs.batched_blocks()[:k], {
            "workload": f"batched (first {k} of the 256 blocks)", "blocks": k}
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
    if name == "paper_scale":
        # the upper range of the paper's length-compatible runs: 1 Gbit key, l = 10%
        b = inputs.single_block(1_000_000_007, 100_000_000, 31, 32)
        return [b], {"workload": f"paper scale n={b.n} m={b.m}", "blocks": 1}
    if name == "paper_scale_3e9":
        # a 3 Gbit key (Fig. 3 runs to 1e10 bits), l = 10%
        b = inputs.single_block(3_000_000_019, 300_000_000, 33, 34)
        return [b], {"workload": f"paper scale n={b.n} m={b.m}", "blocks": 1}
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
    """Device-resident buffers + plans for a list of blocks; one step = all blocks.

    Several blocks run as one batch (pa_batch_plan / pa_batch_run: one persistent
    launch, graph-replayed); a single block runs through pa_plan / pa_hash."""

    def __init__(self, blocks, path: str, device, keys_h=None, seeds_h=None, force_single=False):
        import torch

        import paper_1805_02372_gb300 as pkg
        self.pkg, self.torch = pkg, torch
        self.blocks = blocks
        self.path = path
        self.keys_h = keys_h if keys_h is not None else [b.key() for b in blocks]
        self.seeds_h = seeds_h if seeds_h is not None else [b.seed() for b in blocks]
        t = lambda a: torch.from_numpy(a.view(np.int64)).to(device)
        self.keys = [t(k) for k in self.keys_h]
        self.seeds = [t(s) for s in self.seeds_h]
        self.outs = [torch.zeros((b.m + 63) // 64, dtype=torch.int64, device=device)
                     for b in blocks]
        self.batched = len(blocks) > 1 and not force_single
        self.stream = torch.cuda.current_stream()
        if self.batched:
            self.desc = pkg.BlockList([(b.n, b.m, s, k, o) for b, s, k, o in
                                       zip(blocks, self.seeds, self.keys, self.outs)])
            self.batch = pkg.pa_batch_plan(self.desc, pkg.make_opts(path=path))
            self.plans = None
            self.plan_desc = pkg.pa_batch_describe(self.batch, len(blocks))
        else:
            self.plans = [pkg.Plan(b.n, b.m, path=path) for b in blocks]
            self.plan_desc = [p.desc for p in self.plans]
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

    def paths(self) -> dict:
        out = {}
        for d in self.plan_desc:
            out[d["path_name"]] = out.get(d["path_name"], 0) + 1
        return out

    def e2e(self, steps: int):
        """Same metric through the host-buffer entry points (pinned host memory), copies
        inside the timed region; returns (Gbps, h2d bytes, d2h bytes) per step."""
        torch = self.torch
        pin = lambda a: torch.from_numpy(a.view(np.int64)).pin_memory()
        kh = [pin(k) for k in self.keys_h]
        sh = [pin(s) for s in self.seeds_h]
        oh = [torch.zeros((b.m + 63) // 64, dtype=torch.int64).pin_memory() for b in self.blocks]
        h2d = sum(8 * (k.numel() + s.numel()) for k, s in zip(kh, sh))
        d2h = sum(8 * o.numel() for o in oh)
        if self.batched:
            # descriptors marshalled once (same buffers every step); every step still copies
            # all keys and seeds in and all outputs out
            desc = self.pkg.BlockList([(b.n, b.m, s, k, o) for b, s, k, o in zip(self.blocks, sh, kh, oh)])
            run = lambda: self.pkg.pa_batch_run_host(self.batch, desc, self.stream)
        else:
            run = lambda: [p.hash_host(s, k, o, self.stream)
                           for p, s, k, o in zip(self.plans, sh, kh, oh)]
        run()
        t0 = time.perf_counter()
        for _ in range(steps):
            run()
        dt = (time.perf_counter() - t0) / steps
        for o, w in zip(oh, self.outs):
            if not np.array_equal(o.numpy(), w.cpu().numpy()):
                raise SystemExit("host-buffer entry point disagrees with the device one")
        return self.units / dt / 1e9, h2d, d2h


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


CSRC = "paper_1805_02372_gb300/csrc/"
KERNEL_SOURCES = {
    "direct": [CSRC + "direct.cu", CSRC + "common.cuh"],
    "batch_persistent": [CSRC + "ntt.cu", CSRC + "ntt_defs.cuh", CSRC + "ntt_kernel.cuh",
                         CSRC + "ntt_f29.cu", CSRC + "ntt_f31.cu", CSRC + "ntt_f64.cu",
                         CSRC + "dft.cuh", CSRC + "ntt_field.cuh", CSRC + "tiles.cuh",
                         CSRC + "common.cuh", CSRC + "internal.h"],
    "fft_tile": [CSRC + "fft.cu", CSRC + "dft.cuh", CSRC + "tiles.cuh"],
    "block_mma": [CSRC + "block.cu", CSRC + "common.cuh"],
    "block_tc": [CSRC + "block_tc.cu", CSRC + "common.cuh"],
}

CLOCK_HZ = 2070e6
SMS = 152
# dense FP8 tensor rate: 16384 flops per SM per clock (8192 e4m3 MACs), at the maximum clock
FP8_DERIVED_TFLOPS = SMS * 16384 * CLOCK_HZ / 1e12


def _ntt_ops(descs):
    """8 integer ops per butterfly. A standard tile pair of size N costs 3 (N/2) log2 N + N/2
    butterflies (two forward transforms, one inverse, the pointwise product); a block under
    transform-domain accumulation costs (Q + W + G P) (N/2) log2 N for its Q key, W window
    and G P output transforms (G sums per output tile) plus P Q N products summed."""
    ops = 0.0
    for d in descs:
        if d["path_name"] not in ("ntt31", "ntt64"):
            continue
        k = d["log2_transform"]
        N = 2.0 ** k
        P, Q = d["tiles_out"], d["tiles_in"]
        if d.get("fd"):
            G = d.get("sum_groups") or 1
            ops += 8.0 * ((Q + d["windows"] + G * P) * (N / 2) * k + P * Q * N)
        else:
            ops += 8.0 * P * Q * (3 * (N / 2) * k + N / 2)
    return ops


def algorithmic(kernel: str, blocks, descs):
    """(bound, algorithmic units per step, unit, peak, peak_source) for a kernel."""
    int_alu = SMS * 64 * CLOCK_HZ / 1e12
    int_all = SMS * 128 * CLOCK_HZ / 1e12
    if kernel == "direct":
        # 32 funnel shifts + 32 LOP3 per 32 rows x 32 key bits: m*n/16 integer ops.
        ops = sum(2.0 * b.m * b.n / 32.0 for b, d in zip(blocks, descs)
                  if d["path_name"] == "direct")
        return "alu", ops, "Tops/s", int_alu, "derived: 152 SM x 64 INT32 lanes x 2070 MHz"
    if kernel == "batch_persistent":
        return ("alu", _ntt_ops(descs), "Tops/s", int_all,
                "derived: 152 SM x (64 ALU + 64 FMA-pipe IMAD) lanes x 2070 MHz")
    if kernel == "block_mma":
        ops = sum(2.0 * b.m * (b.n + 8192) for b, d in zip(blocks, descs)
                  if d["path_name"] == "block_int8")
        return "tensor", ops, "Tops/s", 150.8, "measured: legacy mma.sync s8 peak on GB300"
    if kernel == "block_tc":
        # dense FP8 MMA work the kernel performs: M = 128 rows x N = 256 blocks per output
        # tile, over the tile's contraction length n + 128 * 255
        ops = sum(2.0 * 32768 * -(-b.m // 32768) * (b.n + 128 * 255)
                  for b, d in zip(blocks, descs) if d["path_name"] == "block_fp8")
        pk, src = peaks()
        return ("tensor", ops, "TFLOP/s", 2.0 * pk["bf16_tflops"],
                f"{src} bf16 dense x 2 (nominal fp8 / bf16 ratio, 4.5 / 2.25 PFLOP/s); the bf16 "
                f"figure was taken under the power cap (median SM clock in MEASURED_PEAKS), so a "
                f"kernel holding the maximum clock can exceed it: the clock-derived dense FP8 "
                f"peak is {FP8_DERIVED_TFLOPS:.0f} TFLOP/s")
    if kernel == "fft_tile":
        fl = 0.0
        for b, d in zip(blocks, descs):
            if d["path_name"] == "fft":
                N = 2.0 ** d["log2_transform"]
                fl += d["tiles_in"] * d["tiles_out"] * 3 * (N / 2) * d["log2_transform"] * 10
        return ("alu", fl, "TFLOP/s", SMS * 128 * 2 * CLOCK_HZ / 1e12,
                "derived: 152 SM x 128 FP32 lanes x 2 flops x 2070 MHz")
    return None, None, None, None, None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def compulsory_bytes(blocks):
    return sum(8 * ((b.n + 63) // 64 + (b.n + b.m - 1 + 63) // 64 + (b.m + 63) // 64)
               for b in blocks)


def roofline(kt: dict, blocks, descs, steps: int, workload_name: str):
    work = {k: v for k, v in kt.items() if k != "memset"}
    if not work:
        return None
    name, v = max(work.items(), key=lambda kv: kv[1]["total_ms"])
    launches_per_step = max(1.0, v["launches"] / steps)
    per_launch_ms = v["total_ms"] / v["launches"]
    bound, units, unit, peak, src = algorithmic(name, blocks, descs)
    out = {"kernel": name, "launch_ms": per_launch_ms, "launches": v["launches"],
           "share": v["total_ms"] / sum(x["total_ms"] for x in kt.values())}
    if bound is not None and units:
        ach = units / launches_per_step / (per_launch_ms * 1e-3) / 1e12
        out.update({"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                    "frac": ach / peak, "peak_source": src})
        if name == "block_tc":
            out["frac_of_clock_derived_peak"] = ach / FP8_DERIVED_TFLOPS
    pk, psrc = peaks()
    hbm = compulsory_bytes(blocks) / launches_per_step / (per_launch_ms * 1e-3) / 1e9
    out["hbm_compulsory"] = {"achieved_gbs": hbm, "peak_gbs": pk["hbm_gbs"],
                             "frac": hbm / pk["hbm_gbs"], "peak_source": psrc + " (MEASURED_PEAKS)"}
    out["traffic"] = traffic_for(name, workload_name)
    return out


def traffic_for(kernel: str, workload_name: str):
    """Per-launch DRAM bytes from the committed ncu summary, if the kernel is unchanged and
    the figure was taken on this bench workload."""
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
    if ent.get("bench_workload") != workload_name:
        return None
    return ent.get("dram_bytes_per_launch")


# --------------------------------------------------------------------------- CPU oracle

def cpu_oracle_gbps(blocks, rows_per_block: int = 40000, seed: int = 3, max_blocks: int = 256):
    """The oracle as it stands (all host cores), timed on a bounded sample of each block.

    The oracle's full hash of a block is one set-up (seed reversal, key masking) plus m row
    evaluations spread over the cores. Per block it is timed on R/4 and on R rows: the
    difference gives the per-row cost (set-up and thread start cancel), the full-block
    time is set-up + m x per-row, summed over the blocks (a uniform sample of at most
    max_blocks of them, scaled up). Returns (Gbps, cores, description)."""
    import oracle
    rng = np.random.default_rng(seed)
    idx = np.arange(len(blocks))
    if len(idx) > max_blocks:
        idx = rng.choice(idx, max_blocks, replace=False)
    est, measured = 0.0, 0.0
    for i in idx:
        b = blocks[i]
        k, s = b.key(), b.seed()
        # about 2e10 bit products per block sampled (bounded CPU time), at least R rows
        r = max(8, min(b.m, max(rows_per_block, int(2e10 / b.n / len(idx)))))
        r1 = max(1, r // 4)
        rows = rng.integers(0, b.m, r)
        t0 = time.perf_counter()
        oracle.hash_rows(b.n, b.m, s, k, rows[:r1])
        t1 = time.perf_counter()
        oracle.hash_rows(b.n, b.m, s, k, rows)
        t2 = time.perf_counter()
        per_row = max((t2 - t1) - (t1 - t0), 0.0) / (r - r1)
        setup = max((t1 - t0) - per_row * r1, 0.0)
        est += setup + per_row * b.m
        measured += t2 - t0
    est *= len(blocks) / len(idx)
    gbps = sum(b.n for b in blocks) / est / 1e9
    cores = os.cpu_count() or 1
    return gbps, cores, (f"{len(idx)} of {len(blocks)} blocks, each timed on R/4 and R >= "
                         f"{rows_per_block} uniformly drawn output rows ({measured:.1f} s "
                         f"measured); full-block time = set-up + m x per-row time")


# --------------------------------------------------------------------------- main

def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


# Table 1 of the paper: n = 4..128 Mbit, l = 10% of n, TITAN Xp FP32 (context only).
TABLE1_PAPER_GBPS = {4: 1.25, 8: 1.33, 16: 1.37, 32: 1.38, 64: 1.38, 128: 1.35}


def run_table1(args):
    """Table 1 shapes on this GPU: one block per size, m = floor(0.1 n), AUTO path."""
    import torch
    from paper_1805_02372_gb300 import inputs
    device = torch.device("cuda", 0)
    rows = []
    for mbit, paper in TABLE1_PAPER_GBPS.items():
        n = mbit * 1_000_000
        b = inputs.single_block(n, n // 10, 10 + mbit, 11 + mbit)
        r = Runner([b], args.path, device)
        for _ in range(args.warmup):
            r.step()
        ms = timed(r, args.steps, False, r.stream, None)
        exact = check_sampled(r, rows_per_block=32)
        rows.append({"n_mbit": mbit, "m": b.m, "gbps": n / (ms * 1e-3) / 1e9, "ms": ms,
                     "path": r.plan_desc[0]["path_name"], "bit_exact_sampled": exact,
                     "paper_titan_xp_gbps": paper})
        del r
    val = float(np.mean([x["gbps"] for x in rows]))
    print(json.dumps({"metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
                      "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "u64",
                      "data": "synthetic",
                      "config": {"workload": "Table 1 shapes: n = 4..128 Mbit, l = 10% n, "
                                             "one block each (mean Gbps over sizes)"},
                      "sizes": rows}), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    blocks, cfg = workload(args.workload)
    per_step = []
    for _ in range(min(args.warmup, 1)):
        cpu_oracle_gbps(blocks, rows_per_block=64, max_blocks=8)
    for k in range(args.steps):
        g, cores, desc = cpu_oracle_gbps(blocks, rows_per_block=1024, seed=100 + k, max_blocks=64)
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


def serving_probe(rates, count):
    """Continuous-batching server on the serving workload: Poisson arrivals at each rate,
    n log-uniform in [1e5, 1e8], r uniform in [0.01, 0.5], device-resident requests."""
    from paper_1805_02372_gb300 import serve
    out = []
    for i, rate in enumerate(rates):
        reqs = serve.make_requests(count, rate, master=4 + 100 * i)
        st = serve.replay(reqs, slots=3, max_blocks_per_wave=32)
        st["rate_hz"] = rate
        out.append(st)
        del reqs
    return {"workload": "serving: Poisson arrivals, n log-uniform in [1e5, 1e8], r uniform "
                        "in [0.01, 0.5], device-resident keys and seeds, 3 stream slots",
            "requests_per_rate": count, "rates": out}


def timed(runner, steps, flush, stream, scratch):
    import torch
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    torch.cuda.synchronize()
    for a, b in evs:
        if flush:
            scratch.add_(1)
        a.record(stream)
        runner.step()
        b.record(stream)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs) / steps


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default="batched256")
    ap.add_argument("--path", default="auto")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-kernel comparison")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving latency probe")
    ap.add_argument("--serving-rates", default="100,1000",
                    help="comma-separated request rates (req/s) for the serving probe")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "table1":
        return run_table1(args)

    import torch

    from paper_1805_02372_gb300.dist import Group
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    group = Group("nccl", rank, world, device=device) if world > 1 else None

    blocks, cfg = workload(args.workload)
    runner = Runner(blocks, args.path, device)
    stream = runner.stream
    for _ in range(args.warmup):
        runner.step()
    torch.cuda.synchronize()

    in_bytes = sum(8 * (len(k) + len(s)) for k, s in zip(runner.keys_h, runner.seeds_h))
    flush = in_bytes < 2 * L2_BYTES
    scratch = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=device) if flush else None
    if group:
        group.checked_barrier("timed")
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ms = timed(runner, args.steps, flush, stream, scratch)   # graph replay, no tracing
        wall = time.perf_counter() - t0
        # per-kernel CUDA-event durations (eager launches with event pairs)
        runner.profile(True)
        ms_traced = timed(runner, args.steps, flush, stream, scratch)
        runner.profile(False)
    if group:
        ms = group.max(ms)   # the job's step time is the slowest rank's
        torch.distributed.barrier()
    kt = runner.kernel_times()
    exact = check_sampled(runner)
    clocks = clk.summary()
    e2e_gbps, h2d, d2h = runner.e2e(max(3, args.steps // 2))

    units = runner.units * world
    value = units / (ms * 1e-3) / 1e9
    launches = sum(v["launches"] for k, v in kt.items() if k != "memset") // args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": dict(cfg, path=args.path, paths_chosen=runner.paths(),
                       l2="flushed between steps" if flush else "inputs larger than L2",
                       bit_exact_sampled=exact),
        "roofline": roofline(kt, blocks, runner.plan_desc, args.steps, args.workload),
        "e2e": {"value": e2e_gbps * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches * args.steps, "clocks": clocks,
        "kernel_times_ms": {k: round(v["total_ms"] / args.steps, 5) for k, v in kt.items()},
        "ms_per_step_traced": ms_traced, "wall_s": wall,
    }
    if not exact:
        line["error"] = "sampled rows disagree with the oracle"
    if len(blocks) > 1 and not args.no_plain and rank == 0:
        # the plain single-block kernel (direct path), block by block, same blocks
        plain = Runner(blocks, "direct", device, runner.keys_h, runner.seeds_h,
                       force_single=True)
        plain.step()
        pms = timed(plain, 2, flush, stream, scratch)
        line["plain_kernel"] = {"value": runner.units / (pms * 1e-3) / 1e9, "unit": UNIT,
                                "path": "direct, one pa_hash per block", "ms_per_step": pms,
                                "batched_over_plain": value / (runner.units / (pms * 1e-3) / 1e9)}
    if rank == 0 and not args.no_serving:
        rates = [float(r) for r in args.serving_rates.split(",") if r]
        line["serving"] = serving_probe(rates, 60)
        worst = max(r["p99_ms"] for r in line["serving"]["rates"])
        line["p99_latency_ms"] = worst
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, cores, desc = cpu_oracle_gbps(blocks)
        line["cpu_baseline"] = {"value": g, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": desc}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if group:
        group.close()


if __name__ == "__main__":
    main()
