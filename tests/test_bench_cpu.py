"""bench.py's accounting on the CPU: roofline figures, traffic lookup, CPU-baseline sampling.

The GPU runs of bench.py print one JSON line whose roofline, traffic and baseline fields are
computed by these helpers; here they get synthetic kernel times and plan descriptors.
"""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1805_02372_gb300 import inputs  # noqa: E402


def _descs(path, blocks, **extra):
    return [dict({"path_name": path, "log2_transform": 20, "tiles_in": 2, "tiles_out": 1,
                  "fd": 2, "windows": 2}, **extra) for _ in blocks]


def test_roofline_batch_persistent_fields():
    blocks = inputs.batched_blocks()[:4]
    kt = {"batch_persistent": {"launches": 10, "total_ms": 20.0}, "memset": {"launches": 10, "total_ms": 0.1}}
    r = bench.roofline(kt, blocks, _descs("ntt31", blocks), steps=10, workload_name="batched4")
    assert r["kernel"] == "batch_persistent" and r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # achieved = model ops per launch / launch time; one launch per step here
    ops = bench._ntt_ops(_descs("ntt31", blocks))
    assert r["achieved"] == pytest.approx(ops / 2e-3 / 1e12)
    assert r["traffic"] is None  # no committed figure for this workload
    assert 0 < r["hbm_compulsory"]["frac"] < 1


def test_roofline_block_tc_tensor_bound():
    b = inputs.single_block(1_000_000, 500_000)
    kt = {"block_tc": {"launches": 2, "total_ms": 0.6}, "reverse_key": {"launches": 2, "total_ms": 0.01}}
    r = bench.roofline(kt, [b], _descs("block_fp8", [b]), steps=2, workload_name="x")
    flops = 2.0 * 32768 * 16 * (1_000_000 + 128 * 255)
    assert r["bound"] == "tensor" and r["achieved"] == pytest.approx(flops / 0.3e-3 / 1e12)
    assert r["frac_of_clock_derived_peak"] == pytest.approx(r["achieved"] / bench.FP8_DERIVED_TFLOPS)


def test_traffic_lookup_matches_digest_and_workload():
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        tab = json.load(f)
    for kernel, ent in tab.items():
        assert kernel in bench.KERNEL_SOURCES
        # a figure is quoted only for the sources and the bench workload it was taken on
        fresh = ent["source_digest"] == bench._source_digest(bench.KERNEL_SOURCES[kernel])
        want = ent["dram_bytes_per_launch"] if fresh else None
        assert bench.traffic_for(kernel, ent["bench_workload"]) == want
        assert bench.traffic_for(kernel, "another workload") is None


def test_cpu_baseline_sample_is_bounded():
    blocks = [inputs.single_block(20_000, 5_000, 5, 6), inputs.single_block(3_001, 700, 7, 8)]
    g, cores, desc = bench.cpu_oracle_gbps(blocks, rows_per_block=64, max_blocks=2)
    assert g > 0 and cores >= 1 and "2 of 2 blocks" in desc


def test_workloads_named_by_shape():
    for name in ("plain_single", "plain_vs_transform_m250000", "finite_size", "paper_scale",
                 "paper_scale_3e9",
                 "batched8"):
        blocks, cfg = bench.workload(name)
        assert blocks and cfg["blocks"] == len(blocks) and cfg["workload"]


def test_ntt_ops_counts_one_inverse_per_sum():
    # accumulated block: (Q + W + G P) transforms of (N/2) log2 N butterflies plus P Q N
    # summed products, 8 ops each
    d = {"path_name": "ntt31", "log2_transform": 23, "tiles_in": 239, "tiles_out": 24,
         "fd": 1, "windows": 262, "sum_groups": 3}
    N = 2.0 ** 23
    want = 8.0 * ((239 + 262 + 3 * 24) * (N / 2) * 23 + 24 * 239 * N)
    assert bench._ntt_ops([d]) == pytest.approx(want)
    assert bench._ntt_ops([dict(d, sum_groups=1)]) < want
