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


PROBE = {"butterfly_per_s": 5e12, "group28_per_s": 7e12, "group29_per_s": 6e12,
         "muladd_per_s": 4e12, "shift_and_per_s": 9e12}


def test_roofline_batch_persistent_fields():
    blocks = inputs.batched_blocks()[:4]
    kt = {"batch_persistent": {"launches": 10, "total_ms": 20.0}, "memset": {"launches": 10, "total_ms": 0.1}}
    # two blocks over the 28-bit prime, one over the 29-bit, one over the 64-bit
    descs = _descs("ntt31", blocks, prime_bits=28)
    descs[2] = dict(descs[2], prime_bits=29)
    descs[3] = dict(descs[3], prime_bits=64, path_name="ntt64")
    r = bench.roofline(kt, blocks, descs, steps=10, workload_name="batched4", probe=PROBE)
    assert r["kernel"] == "batch_persistent" and r["bound"] == "alu" and r["unit"] == "Tops/s"
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    # achieved = model ops per launch / launch time; one launch per step here
    bfly, prod = bench.ntt_work(descs)
    assert set(bfly) == {28, 29, 64} and bfly[28] == pytest.approx(2 * bfly[29])
    assert r["achieved"] == pytest.approx(bench.OPS_PER_BFLY * (sum(bfly.values()) + prod) / 2e-3 / 1e12)
    # the fraction is the time the work takes at the measured peaks over the launch time:
    # each field's butterflies at its group rate (the 64-bit field at the single-butterfly rate)
    t_peak = (bfly[28] / PROBE["group28_per_s"] + bfly[29] / PROBE["group29_per_s"] +
              bfly[64] / PROBE["butterfly_per_s"] + prod / PROBE["muladd_per_s"])
    assert r["frac"] == pytest.approx(t_peak / 2e-3)
    assert "measured in this run" in r["peak_source"]
    assert r["traffic"] is None  # no committed figure for this workload
    assert 0 < r["hbm_compulsory"]["frac"] < 1


def test_roofline_without_probe_reports_no_fraction():
    blocks = inputs.batched_blocks()[:2]
    kt = {"batch_persistent": {"launches": 2, "total_ms": 2.0}}
    r = bench.roofline(kt, blocks, _descs("ntt31", blocks), steps=2, workload_name="x")
    assert "frac" not in r and r["hbm_compulsory"]["frac"] > 0


def test_roofline_direct_against_shift_and_peak():
    b = inputs.single_block(1_000_000, 500_000)
    kt = {"direct": {"launches": 4, "total_ms": 8.0}}
    r = bench.roofline(kt, [b], _descs("direct", [b]), steps=4, workload_name="x", probe=PROBE)
    ops = b.m * b.n / 32.0
    assert r["frac"] == pytest.approx(ops / PROBE["shift_and_per_s"] / 2e-3)


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


def test_cpu_baseline_times_whole_blocks():
    blocks = [inputs.single_block(20_000, 5_000, 5, 6), inputs.single_block(3_001, 700, 7, 8)]
    g, k, t, bits, th = bench.cpu_oracle_measured(blocks, budget_s=60.0)
    assert k == 2 and bits == 23_001 and t > 0 and th >= 1
    assert g == pytest.approx(bits / t / 1e9)
    # the budget bounds the sample: with none left after the first block, one block is timed
    g1, k1, _, bits1, _ = bench.cpu_oracle_measured(blocks, budget_s=0.0, threads=1, order=[1, 0])
    assert k1 == 1 and bits1 == 3_001 and g1 > 0


def test_golden_digests_for_batched_prefixes():
    d = bench.golden_digests("batched8")
    assert d is not None and len(d) == 8 and all(len(x) == 64 for x in d)
    assert bench.golden_digests("plain_single") is None


def test_workloads_named_by_shape():
    for name in ("plain_single", "plain_vs_transform_m250000", "finite_size", "paper_scale",
                 "paper_scale_3e9",
                 "batched8"):
        blocks, cfg = bench.workload(name)
        assert blocks and cfg["blocks"] == len(blocks) and cfg["workload"]


def test_ntt_work_counts_one_inverse_per_sum():
    # accumulated block: (Q + W + G P) transforms of (N/2) log2 N butterflies plus P Q N
    # summed products
    d = {"path_name": "ntt31", "log2_transform": 23, "tiles_in": 239, "tiles_out": 24,
         "fd": 1, "windows": 262, "sum_groups": 3}
    N = 2.0 ** 23
    bfly, prod = bench.ntt_work([d])
    assert bfly[29] == pytest.approx((239 + 262 + 3 * 24) * (N / 2) * 23)
    assert prod == pytest.approx(24 * 239 * N)
    assert bench.ntt_work([dict(d, sum_groups=1)])[0][29] < bfly[29]
    # a standard tile pair: two forward transforms, one inverse, N pointwise products
    p = {"path_name": "ntt31", "log2_transform": 20, "tiles_in": 3, "tiles_out": 2, "fd": 0,
         "windows": 0}
    b2, p2 = bench.ntt_work([dict(p, prime_bits=28)])
    assert b2 == {28: pytest.approx(6 * 3 * (2.0 ** 19) * 20)} and p2 == pytest.approx(6 * 2.0 ** 20)
