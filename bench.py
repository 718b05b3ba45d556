#!/usr/bin/env python3
"""Throughput bench of the GB300 Toeplitz hash (privacy amplification, arXiv 1805.02372).

One step = one pass of the whole hot path over the workload's blocks: plan lookup,
the decomposition into tiles, the kernels, the XOR merge, packed output. Inputs are
seeded synthetic uniform bits, resident in HBM before the timed region; the metric
is input-key Gbps (sum of n over the blocks / device time, Mbit = 10^6 bits as in
Table 1), bit-exact against the CPU oracle (checked on sampled rows every run).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                       [--path auto|direct|ntt64|ntt31|fft|block_int8|block_fp8]
                       [--impl ours|reference] [--quick]
Under torchrun every rank runs the same workload on its own GPU (independent
blocks: weak scaling, no data-path collective); rank 0 prints one JSON line.

Besides the headline (the batched workload on the autotuned path), rank 0 adds to the
same line: the plain single-block kernel on the same blocks, the batched workload with
each path forced, the single-block workloads on several paths, Table 1's shapes, the
serving workload at five request rates, the measured issue-rate peaks the roofline
fractions are taken against, and the CPU oracle timed on whole blocks (all cores and
one core). ``--quick`` leaves those out.
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
    if name == "paper_scale_1e10":
        # the top of Fig. 3's range, l = 10%: segmented sums in a fixed workspace
        b = inputs.single_block(10_000_000_019, 1_000_000_000, 35, 36)
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
        inside the timed region; returns (Gbps, h2d bytes, d2h bytes, serial Gbps, how) per
        step. Batched: every step copies all keys and seeds in and all outputs out; two
        batches of the same plan alternate on two streams (pa_batch_run_host_async, copies
        by the copy engines), so one step's copies run while the other step computes. The
        serial figure runs one synchronous pa_batch_run_host per step."""
        torch = self.torch
        pin = lambda a: torch.from_numpy(a.view(np.int64)).pin_memory()
        kh = [pin(k) for k in self.keys_h]
        sh = [pin(s) for s in self.seeds_h]
        zeros = lambda: [torch.zeros((b.m + 63) // 64, dtype=torch.int64).pin_memory() for b in self.blocks]
        oh = zeros()
        h2d = sum(8 * (k.numel() + s.numel()) for k, s in zip(kh, sh))
        d2h = sum(8 * o.numel() for o in oh)

        def timed(run):
            run()
            t0 = time.perf_counter()
            for _ in range(steps):
                run()
            return (time.perf_counter() - t0) / steps

        def check(outs):
            for o, w in zip(outs, self.outs):
                if not np.array_equal(o.numpy(), w.cpu().numpy()):
                    raise SystemExit("host-buffer entry point disagrees with the device one")

        if not self.batched:
            dt = timed(lambda: [p.hash_host(s, k, o, self.stream)
                                for p, s, k, o in zip(self.plans, sh, kh, oh)])
            check(oh)
            g = self.units / dt / 1e9
            return g, h2d, d2h, g, "one synchronous pa_hash_host per block and step"
        # descriptors marshalled once (same buffers every step)
        desc = self.pkg.BlockList([(b.n, b.m, s, k, o) for b, s, k, o in zip(self.blocks, sh, kh, oh)])
        serial = timed(lambda: self.pkg.pa_batch_run_host(self.batch, desc, self.stream))
        check(oh)
        oh2, oh3 = zeros(), zeros()
        d2 = self.pkg.BlockList([(b.n, b.m, s, k, o) for b, s, k, o in zip(self.blocks, sh, kh, oh2)])
        d3 = self.pkg.BlockList([(b.n, b.m, s, k, o) for b, s, k, o in zip(self.blocks, sh, kh, oh3)])
        b2 = self.pkg.pa_batch_plan(self.desc, self.pkg.make_opts(path=self.path))
        streams = [torch.cuda.Stream(), torch.cuda.Stream()]
        pairs = [(self.batch, d2, streams[0]), (b2, d3, streams[1])]

        def piped(k):
            for i in range(k):
                b, d, st = pairs[i % 2]
                self.pkg.pa_batch_run_host_async(b, d, st)
            for st in streams:
                st.synchronize()

        piped(2)
        t0 = time.perf_counter()
        piped(steps)
        dt = (time.perf_counter() - t0) / steps
        for b, _, st in pairs:
            self.pkg.pa_batch_get_report(b, st)
        check(oh2)
        check(oh3)
        self.pkg.pa_batch_destroy(b2)
        return (self.units / dt / 1e9, h2d, d2h, self.units / serial / 1e9,
                "two batches of the same plan alternating on two streams (pa_batch_run_host_async: "
                "all keys and seeds copied in and all outputs out every step, by the copy engines, "
                "one step's copies overlapping the other step's kernels)")


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
                         CSRC + "ntt_f28.cu", CSRC + "ntt_f29.cu", CSRC + "ntt_f31.cu",
                         CSRC + "ntt_f64.cu",
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
# integer operations per butterfly and per field multiply-add, the counting unit of the
# achieved / peak figures in Tops/s (the fraction itself is a ratio of times and does
# not depend on it)
OPS_PER_BFLY = 8


def ntt_work(descs):
    """(butterflies by prime bits, multiply-adds) of the NTT blocks: a standard tile pair of
    size N is two forward transforms and one inverse, (N/2) log2 N butterflies each, and N
    pointwise products; a block under transform-domain accumulation computes its Q key, W
    window and G P output transforms once (G sums per output tile) and sums P Q N products."""
    bfly = {}
    prod = 0.0
    for d in descs:
        if d["path_name"] not in ("ntt31", "ntt64"):
            continue
        pb = d.get("prime_bits") or 29
        k = d["log2_transform"]
        N = 2.0 ** k
        P, Q = d["tiles_out"], d["tiles_in"]
        b = 0.0
        if d.get("fd"):
            # segmented sums recompute the key spectra once per output slice; `windows` and
            # `sum_groups` count every segment's
            G = d.get("sum_groups") or 1
            so = d.get("seg_out") or P
            keys = Q * -(-P // so)
            b += (keys + d["windows"] + G * P) * (N / 2) * k
            if d.get("outer_log2"):
                # sums as convolutions over the tile index: per (group, output slice) three
                # T-point transforms and T products for every bin
                T, lt = 2.0 ** d["outer_log2"], d["outer_log2"]
                conv = G * -(-P // so) * -(-so // d["outer_slice"])
                b += conv * N * 3 * (T / 2) * lt
                prod += conv * N * T
            else:
                prod += P * Q * N
        else:
            b += P * Q * 3 * (N / 2) * k
            prod += P * Q * N
        bfly[pb] = bfly.get(pb, 0.0) + b
    return bfly, prod


def spectra_elements(descs):
    """Transform-domain elements the NTT blocks' spectra hold over a step (every transform's
    N): the unit the persistent launch's DRAM traffic grows with, used to scale a traffic
    figure captured on a subset of the blocks to the whole launch."""
    tot = 0.0
    for d in descs:
        if d["path_name"] not in ("ntt31", "ntt64"):
            continue
        N = 2.0 ** d["log2_transform"]
        P, Q = d["tiles_out"], d["tiles_in"]
        if d.get("fd"):
            keys = Q * -(-P // (d.get("seg_out") or P))
            tot += (keys + d["windows"] + (d.get("sum_groups") or 1) * P) * N
        else:
            tot += 3 * P * Q * N
    return tot


def algorithmic(kernel: str, blocks, descs, probe):
    """(bound, algorithmic ops per step, unit, seconds those ops take at the peak per step,
    peak_source) for a kernel; `probe` holds the issue-rate peaks measured in this run."""
    if kernel == "direct":
        # one shift-and-accumulate per (row, 32 key bits): m n / 32 of them
        ops = sum(b.m * b.n / 32.0 for b, d in zip(blocks, descs) if d["path_name"] == "direct")
        if not probe:
            return None, None, None, None, None
        return ("alu", ops, "Tops/s", ops / probe["shift_and_per_s"],
                f"measured in this run: pa_probe_peak(PA_PEAK_SHIFT_AND) = "
                f"{probe['shift_and_per_s'] / 1e12:.2f} T shift-and-accumulates/s")
    if kernel == "batch_persistent":
        bfly, prod = ntt_work(descs)
        if not probe:
            return None, None, None, None, None
        # butterflies at the measured rate of their field's radix-16 groups (the kernel's
        # rounds; fields without a group probe at the single-butterfly rate)
        rate = {28: probe["group28_per_s"], 29: probe["group29_per_s"]}
        t_peak = sum(b / rate.get(pb, probe["butterfly_per_s"]) for pb, b in bfly.items())
        t_peak += prod / probe["muladd_per_s"]
        nb = sum(bfly.values())
        fields = ", ".join(f"{b:.4g} over the {pb}-bit prime" for pb, b in sorted(bfly.items()))
        return ("alu", OPS_PER_BFLY * (nb + prod), "Tops/s", t_peak,
                f"measured in this run: pa_probe_peak radix-16 butterfly groups of the 28-bit "
                f"field {probe['group28_per_s'] / 1e12:.3f} T/s and of the 29-bit field "
                f"{probe['group29_per_s'] / 1e12:.3f} T/s (the kernel's rounds: lazy reduction "
                f"schedule, twiddles from shared memory, values in registers, on all SMs), "
                f"multiply-adds {probe['muladd_per_s'] / 1e12:.3f} T/s; peak time = butterflies "
                f"({fields}) / their field's rate + {prod:.4g} multiply-adds / that; "
                f"{OPS_PER_BFLY} ops per butterfly or multiply-add")
    if kernel == "block_mma":
        ops = sum(2.0 * b.m * (b.n + 8192) for b, d in zip(blocks, descs)
                  if d["path_name"] == "block_int8")
        if not probe:
            return None, None, None, None, None
        return ("tensor", ops, "Tops/s", ops / (2.0 * probe["mma_s8_macs_per_s"]),
                f"measured in this run: pa_probe_peak(PA_PEAK_MMA_S8) = "
                f"{2.0 * probe['mma_s8_macs_per_s'] / 1e12:.1f} Top/s (legacy mma.sync s8)")
    if kernel == "block_tc":
        # dense FP8 MMA work the kernel performs: M = 128 rows x N = 256 blocks per output
        # tile, over the tile's contraction length n + 128 * 255
        ops = sum(2.0 * 32768 * -(-b.m // 32768) * (b.n + 128 * 255)
                  for b, d in zip(blocks, descs) if d["path_name"] == "block_fp8")
        pk, src = peaks()
        return ("tensor", ops, "TFLOP/s", ops / (2.0 * pk["bf16_tflops"] * 1e12),
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
        peak = SMS * 128 * 2 * CLOCK_HZ
        return ("alu", fl, "TFLOP/s", fl / peak,
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


def roofline(kt: dict, blocks, descs, steps: int, workload_name: str, probe=None):
    work = {k: v for k, v in kt.items() if k != "memset"}
    if not work:
        return None
    name, v = max(work.items(), key=lambda kv: kv[1]["total_ms"])
    launches_per_step = max(1.0, v["launches"] / steps)
    per_launch_ms = v["total_ms"] / v["launches"]
    bound, units, unit, t_peak, src = algorithmic(name, blocks, descs, probe)
    out = {"kernel": name, "launch_ms": per_launch_ms, "launches": v["launches"],
           "share": v["total_ms"] / sum(x["total_ms"] for x in kt.values())}
    if bound is not None and units:
        t_launch = per_launch_ms * 1e-3 * launches_per_step  # kernel seconds per step
        ach = units / t_launch / 1e12
        peak = units / t_peak / 1e12
        out.update({"bound": bound, "achieved": ach, "peak": peak, "unit": unit,
                    "frac": ach / peak, "peak_source": src})
        if name == "block_tc":
            out["frac_of_clock_derived_peak"] = ach / FP8_DERIVED_TFLOPS
    pk, psrc = peaks()
    hbm = compulsory_bytes(blocks) / launches_per_step / (per_launch_ms * 1e-3) / 1e9
    out["hbm_compulsory"] = {"achieved_gbs": hbm, "peak_gbs": pk["hbm_gbs"],
                             "frac": hbm / pk["hbm_gbs"], "peak_source": psrc + " (MEASURED_PEAKS)",
                             "bytes_per_step": compulsory_bytes(blocks)}
    out["traffic"] = traffic_for(name, workload_name)
    if name == "batch_persistent":
        out["spectra_elements_per_launch"] = spectra_elements(descs) / launches_per_step
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

def cpu_oracle_measured(blocks, budget_s: float = 20.0, threads: int | None = None,
                        order=None, seed: int = 3):
    """The oracle as it stands, timed on WHOLE blocks: blocks are hashed in full, in a
    seeded random order (or the given order), until `budget_s` seconds of oracle time have
    passed (the block running then is finished). Returns (Gbps over the blocks hashed,
    blocks hashed, oracle seconds, key bits, threads). Key and seed generation is not
    timed."""
    import oracle
    if order is None:
        order = np.random.default_rng(seed).permutation(len(blocks))
    th = threads or oracle.default_threads()
    spent, bits, done = 0.0, 0, 0
    for i in order:
        if done and spent >= budget_s:
            break
        b = blocks[int(i)]
        k, s_ = b.key(), b.seed()
        t0 = time.perf_counter()
        oracle.hash_full(b.n, b.m, s_, k, threads=th)
        spent += time.perf_counter() - t0
        bits += b.n
        done += 1
    return bits / spent / 1e9, done, spent, bits, th


def cpu_baseline(blocks):
    """All host cores on a random sample of whole blocks (about 20 s), and one core on the
    cheapest blocks (by m n, about 8 s)."""
    g, k, t, _, th = cpu_oracle_measured(blocks, budget_s=20.0)
    cheap = np.argsort([b.m * b.n for b in blocks], kind="stable")
    g1, k1, t1, _, _ = cpu_oracle_measured(blocks, budget_s=8.0, threads=1, order=cheap)
    return {"value": g, "unit": UNIT, "cores": th, "kind": "oracle",
            "sample": f"{k} of {len(blocks)} blocks hashed in full (seeded random order, "
                      f"{t:.1f} s measured on {th} threads); Gbps = their key bits / that time",
            "single_core": {"value": g1, "unit": UNIT, "cores": 1,
                            "sample": f"the {k1} blocks of least m n hashed in full on one "
                                      f"thread ({t1:.1f} s measured)"}}


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
    """The reference arm: the CPU oracle as it stands, on the host cores. Each step hashes
    in full the next blocks of a seeded random order of the workload's blocks until about
    two seconds of oracle time have passed; the value is the key bits of the blocks timed
    over the time they took, and ms_per_step is the measured mean step time."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    blocks, cfg = workload(args.workload)
    order = np.random.default_rng(11).permutation(len(blocks))
    pos = 0

    def one_step():
        nonlocal pos
        t_step, bits_step = 0.0, 0
        while t_step < 2.0:
            i = order[pos % len(order)]
            pos += 1
            _, _, t, bits, th = cpu_oracle_measured(blocks, budget_s=0.0, order=[i])
            t_step += t
            bits_step += bits
        return t_step, bits_step, th

    tot_t, tot_bits, th, per_step = 0.0, 0, oracle.default_threads(), []
    for k in range(args.warmup + args.steps):
        t_step, bits_step, th = one_step()
        if k >= args.warmup:
            tot_t += t_step
            tot_bits += bits_step
            per_step.append(t_step)
    val = tot_bits / tot_t / 1e9
    desc = (f"each step hashes whole blocks in full (next blocks of a seeded random order, "
            f"at least 2 s of oracle time per step); {args.steps} timed steps covered "
            f"{tot_bits / 1e6:.1f} Mbit in {tot_t:.1f} s on {th} threads")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": float(np.mean(per_step)) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": dict(cfg, sample="whole blocks per step, see cpu_baseline"),
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": th, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


SERVING_RATES = (10.0, 100.0, 500.0, 1000.0, 2000.0)


def serving_probe(rates, count):
    """Continuous-batching server on the serving workload: Poisson arrivals at each rate,
    n log-uniform in [1e5, 1e8], r uniform in [0.01, 0.5], device-resident requests. The
    same `count` requests (shapes and buffers) are replayed at every rate, their arrival
    times rescaled. The saturation rate is the lowest rate whose sustained throughput
    falls below 0.9 of the offered load or whose late arrivals wait three times longer
    than the early ones (the queue grows)."""
    import torch

    from paper_1805_02372_gb300 import serve
    base = serve.make_requests(count, 1000.0)
    out = []
    for rate in rates:
        st = serve.replay(serve.at_rate(base, rate, 1000.0), slots=3, max_blocks_per_wave=32,
                          timeout_s=60.0 + 3.0 * count / rate)
        st["rate_hz"] = rate
        out.append(st)
    sat = next((r["rate_hz"] for r in out
                if r["sustained_gbps"] < 0.9 * r["offered_gbps"] or r["latency_drift"] > 3.0),
               None)
    del base
    torch.cuda.empty_cache()
    return {"workload": "serving: Poisson arrivals, n log-uniform in [1e5, 1e8], r uniform "
                        "in [0.01, 0.5], device-resident keys and seeds, 3 stream slots, "
                        "at most 32 requests per wave",
            "requests_per_rate": count, "rates": out, "saturation_rate_hz": sat,
            "saturation_rule": "lowest rate with sustained < 0.9 offered or latency drift > 3"}


def probe_peaks():
    """Issue-rate peaks of this GPU for the integer paths' operations (pa_probe_peak)."""
    from paper_1805_02372_gb300 import binding
    b, bms = binding.pa_probe_peak(binding.PA_PEAK_NTT_BUTTERFLY)
    g28, g28ms = binding.pa_probe_peak(binding.PA_PEAK_NTT_GROUP28)
    g29, g29ms = binding.pa_probe_peak(binding.PA_PEAK_NTT_GROUP29)
    ma, mms = binding.pa_probe_peak(binding.PA_PEAK_NTT_MULADD)
    sa, sms = binding.pa_probe_peak(binding.PA_PEAK_SHIFT_AND)
    s8, s8ms = binding.pa_probe_peak(binding.PA_PEAK_MMA_S8)
    b1, b1ms = binding.pa_probe_peak(binding.PA_PEAK_MMA_B1)
    return {"butterfly_per_s": b, "group28_per_s": g28, "group29_per_s": g29,
            "muladd_per_s": ma, "shift_and_per_s": sa,
            "mma_s8_macs_per_s": s8, "mma_b1_and_popc_per_s": b1,
            "launch_ms": {"butterfly": bms, "group28": g28ms, "group29": g29ms, "muladd": mms,
                          "shift_and": sms, "mma_s8": s8ms, "mma_b1": b1ms},
            "what": "29-bit-field single lazy butterfly; radix-16 forward and inverse groups of "
                    "the 28- and 29-bit fields as the NTT rounds run them (twiddles from shared "
                    "memory); 29-bit-field multiply-add; funnel-shift AND-XOR; mma.sync "
                    "m16n8k32 s8 and m16n8k256 b1 AND-POPC: chains in registers on every SM, "
                    "fastest of three ~20 ms launches after a warm-up"}


def binary_mma_record(probe, fp8_rec):
    """The block contraction's dense forms compared in bit products per second: the
    binary mma.sync (one AND per bit product), the INT8 mma.sync (one MAC per bit product),
    the tcgen05 FP8 path (measured on the batched workload: one MAC per bit product) and
    the direct kernel's shift-and-accumulate (32 bit products each)."""
    out = {"b1_mma_bit_products_per_s": probe["mma_b1_and_popc_per_s"],
           "s8_mma_bit_products_per_s": probe["mma_s8_macs_per_s"],
           "direct_bit_products_per_s": 32.0 * probe["shift_and_per_s"]}
    if fp8_rec and "roofline" in fp8_rec:
        out["fp8_tcgen05_bit_products_per_s"] = fp8_rec["roofline"]["achieved"] * 1e12 / 2.0
    return out


# --------------------------------------------------------------------------- full-output checks

def _sha(words) -> str:
    return hashlib.sha256(np.ascontiguousarray(words, dtype="<u8").tobytes()).hexdigest()


def golden_digests(workload_name: str):
    """SHA-256 of the oracle's full output per block, from the committed golden files
    (written by tests/golden/make_golden.py, which calls only the oracle), or None."""
    gd = os.path.join(ROOT, "tests", "golden")
    try:
        if workload_name.startswith("batched"):
            with open(os.path.join(gd, "batched256.json")) as f:
                d = [b["sha256"] for b in json.load(f)["blocks"]]
            k = 256 if workload_name == "batched256" else int(workload_name[len("batched"):])
            return d[:k]
        if workload_name == "finite_size":
            with open(os.path.join(gd, "finite_size.json")) as f:
                return [json.load(f)["sha256"]]
    except (OSError, ValueError, KeyError):
        return None
    return None


def check_full(runner, digests) -> bool | None:
    """Every block's whole output against its stored oracle digest (None: no digests)."""
    if not digests:
        return None
    return all(_sha(o.cpu().numpy().view(np.uint64)) == d for o, d in zip(runner.outs, digests))


# --------------------------------------------------------------------------- sub-records

def run_record(blocks, path, device, steps, flush, scratch, probe, workload_name,
               keys_h=None, seeds_h=None, want=None, digests=None):
    """Time one workload on one path (warm-up, `steps` timed steps, then a traced pass for
    the roofline) and check its output; returns a compact record."""
    import torch
    try:
        r = Runner(blocks, path, device, keys_h, seeds_h)
    except Exception as e:  # a forced path that cannot take these sizes
        return {"path": path, "unsupported": str(e)[:160]}
    r.step()
    torch.cuda.synchronize()
    ms = timed(r, steps, flush, r.stream, scratch)
    r.profile(True)
    timed(r, 1, flush, r.stream, scratch)
    r.profile(False)
    kt = r.kernel_times()
    rec = {"path": path, "paths_chosen": r.paths(), "ms_per_step": ms,
           "gbps": r.units / (ms * 1e-3) / 1e9}
    rf = roofline(kt, blocks, r.plan_desc, 1, workload_name, probe)
    if rf:
        rec["roofline"] = {k: rf[k] for k in ("kernel", "bound", "achieved", "peak", "unit",
                                              "frac") if k in rf}
    if want is not None:
        rec["bit_exact_full"] = all(np.array_equal(o.cpu().numpy().view(np.uint64), w)
                                    for o, w in zip(r.outs, want))
    elif digests:
        rec["bit_exact_full"] = check_full(r, digests)
    else:
        rec["bit_exact_sampled"] = check_sampled(r, rows_per_block=32)
    del r
    torch.cuda.empty_cache()
    return rec


def batched_paths(blocks, keys_h, seeds_h, device, flush, scratch, probe, plain_gbps, digests):
    """The batched workload with every path forced for all blocks (the benchmark spec: the FP32 /
    INT8 / FP8 batched paths against the plain single-block kernel)."""
    out = {}
    for path in ("ntt31", "ntt64", "block_fp8", "direct", "block_int8", "fft"):
        rec = run_record(blocks, path, device, 2, flush, scratch, probe, "batched_" + path,
                         keys_h, seeds_h, digests=digests)
        if "gbps" in rec and plain_gbps:
            rec["over_plain_kernel"] = rec["gbps"] / plain_gbps
        if path == "block_fp8" and "roofline" in rec:
            rec["tensor_pipe_util_of_clock_derived_peak"] = (
                rec["roofline"]["achieved"] / FP8_DERIVED_TFLOPS)
        out[path] = rec
    return out


def config_records(device, flush, scratch, probe):
    """The single-block workloads (plain single block, plain vs transform, finite size) on
    several paths, each output checked in full against the oracle (the finite-size block
    against its stored digest)."""
    import oracle
    from paper_1805_02372_gb300 import inputs
    out = []
    cases = [("plain_single", inputs.PLAIN_SINGLE,
              ("auto", "direct", "ntt31", "ntt64", "fft", "block_int8", "block_fp8"))]
    for b in inputs.PLAIN_VS_TRANSFORM:
        cases.append((f"plain_vs_transform_m{b.m}", b,
                      ("auto", "direct", "ntt31", "ntt64", "fft", "block_int8", "block_fp8")))
    cases.append(("finite_size", inputs.FINITE_SIZE,
                  ("auto", "ntt31", "ntt64", "block_fp8", "direct")))
    for name, b, paths in cases:
        k, s_ = b.key(), b.seed()
        digests = golden_digests(name)
        want = None if name == "finite_size" else [oracle.hash_full(b.n, b.m, s_, k)]
        recs = {}
        for path in paths:
            recs[path] = run_record([b], path, device, 2 if b.n * b.m > 1e14 else 5, flush,
                                    scratch, probe, name, [k], [s_], want=want, digests=digests)
        out.append({"workload": name, "n": b.n, "m": b.m, "paths": recs})
    return out


def table1_records(device, flush, scratch, probe):
    """Table 1's shapes: n = 4..128 Mbit, m = floor(n / 10), one block each, AUTO path."""
    from paper_1805_02372_gb300 import inputs
    rows = []
    for mbit, paper in TABLE1_PAPER_GBPS.items():
        n = mbit * 1_000_000
        b = inputs.single_block(n, n // 10, 10 + mbit, 11 + mbit)
        rec = run_record([b], "auto", device, 5, flush, scratch, probe, f"table1_{mbit}")
        rec.update({"n_mbit": mbit, "m": b.m, "paper_titan_xp_gbps": paper})
        rows.append(rec)
    return rows


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
    ap.add_argument("--quick", action="store_true",
                    help="headline only: no sub-records, serving, probes or CPU baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-kernel comparison")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving latency probe")
    ap.add_argument("--serving-rates", default=",".join(str(int(r)) for r in SERVING_RATES),
                    help="comma-separated request rates (req/s) for the serving probe")
    ap.add_argument("--serving-requests", type=int, default=500)
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
    probe = None
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ms = timed(runner, args.steps, flush, stream, scratch)   # graph replay, no tracing
        wall = time.perf_counter() - t0
        # per-kernel CUDA-event durations (eager launches with event pairs)
        runner.profile(True)
        ms_traced = timed(runner, args.steps, flush, stream, scratch)
        runner.profile(False)
        if rank == 0 and not args.quick:
            probe = probe_peaks()  # same clock window as the timed steps
    if group:
        ms = group.max(ms)   # the job's step time is the slowest rank's
        torch.distributed.barrier()
    kt = runner.kernel_times()
    digests = golden_digests(args.workload)
    exact_full = check_full(runner, digests)
    exact = check_sampled(runner) if exact_full is None else exact_full
    clocks = clk.summary()
    e2e_gbps, h2d, d2h, e2e_serial, e2e_how = runner.e2e(max(3, args.steps // 2))

    units = runner.units * world
    value = units / (ms * 1e-3) / 1e9
    launches = sum(v["launches"] for k, v in kt.items() if k != "memset") // args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": dict(cfg, path=args.path, paths_chosen=runner.paths(),
                       l2="flushed between steps" if flush else "inputs larger than L2",
                       **({"bit_exact_full": exact_full} if exact_full is not None
                          else {"bit_exact_sampled": exact})),
        "roofline": roofline(kt, blocks, runner.plan_desc, args.steps, args.workload, probe),
        "e2e": {"value": e2e_gbps * world, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "serial_value": e2e_serial * world, "how": e2e_how},
        "gpu_launches": launches * args.steps, "clocks": clocks,
        "kernel_times_ms": {k: round(v["total_ms"] / args.steps, 5) for k, v in kt.items()},
        "ms_per_step_traced": ms_traced, "wall_s": wall,
    }
    if probe:
        line["probe_peaks"] = probe
    if not exact:
        line["error"] = "outputs disagree with the oracle"
    keys_h, seeds_h = runner.keys_h, runner.seeds_h
    plain_gbps = None
    extras = rank == 0 and not args.quick
    if len(blocks) > 1 and not args.no_plain and rank == 0:
        # the plain single-block kernel (direct path), block by block, same blocks
        plain = Runner(blocks, "direct", device, keys_h, seeds_h, force_single=True)
        plain.step()
        pms = timed(plain, 2, flush, stream, scratch)
        plain_gbps = runner.units / (pms * 1e-3) / 1e9
        line["plain_kernel"] = {"value": plain_gbps, "unit": UNIT,
                                "path": "direct, one pa_hash per block", "ms_per_step": pms,
                                "batched_over_plain": value / plain_gbps}
        del plain
    del runner
    torch.cuda.empty_cache()
    if extras and len(blocks) > 1:
        line["paths_batched"] = batched_paths(blocks, keys_h, seeds_h, device, flush, scratch,
                                              probe, plain_gbps, digests)
        line["binary_mma"] = binary_mma_record(probe, line["paths_batched"].get("block_fp8"))
    if extras and args.workload == "batched256":
        line["configs"] = config_records(device, flush, scratch, probe)
        line["table1"] = table1_records(device, flush, scratch, probe)
    if extras and not args.no_serving:
        rates = [float(r) for r in args.serving_rates.split(",") if r]
        line["serving"] = serving_probe(rates, args.serving_requests)
        line["p99_latency_ms"] = max(r["p99_ms"] for r in line["serving"]["rates"])
    if extras and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(blocks)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if group:
        group.close()


if __name__ == "__main__":
    main()
