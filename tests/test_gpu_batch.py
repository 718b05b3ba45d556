"""Batched hashing: many blocks of uneven n and m in one persistent launch (graph-replayed).

Each block's bits must equal the oracle's, and equal the same block hashed alone.
"""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle
import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding, inputs
from gpu_util import dev, host

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))

MIXED = [(100_003, 25_000), (1, 1), (64, 70_001), (4_097, 4_095), (1_000_000, 10_000),
         (262_145, 131_071), (2_000_003, 900_001), (33_333, 33_333), (1_048_577, 3),
         (150_000, 1_500), (700_001, 350_000), (5, 900)]


def _blocks(shapes, salt=0):
    bl = [inputs.single_block(n, m, 1000 + 2 * i + salt, 1001 + 2 * i + salt)
          for i, (n, m) in enumerate(shapes)]
    keys = [b.key() for b in bl]
    seeds = [b.seed() for b in bl]
    return bl, keys, seeds


def _run_batch(bl, keys, seeds, opts=None, runs=2):
    import torch
    kd = [dev(k) for k in keys]
    sd = [dev(s) for s in seeds]
    od = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in bl]
    desc = [(b.n, b.m, s, k, o) for b, s, k, o in zip(bl, sd, kd, od)]
    batch = pkg.pa_batch_plan(desc, opts)
    reps = [pkg.pa_batch_run(batch, desc, report=True) for _ in range(runs)]
    paths = [d["path_name"] for d in pkg.pa_batch_describe(batch, len(bl))]
    pkg.pa_batch_destroy(batch)
    return [host(o) for o in od], reps, paths


@pytest.mark.parametrize("path", ["auto", "ntt31", "ntt64", "direct", "fft", "block_int8",
                                  "block_fp8"])
def test_mixed_batch_matches_oracle(path):
    bl, keys, seeds = _blocks(MIXED)
    if path == "fft":  # keep the FP tile count modest
        bl, keys, seeds = _blocks([s for s in MIXED if s[0] * s[1] < 5e10])
    outs, reps, paths = _run_batch(bl, keys, seeds, binding.make_opts(path=path))
    for b, k, s, y in zip(bl, keys, seeds, outs):
        assert np.array_equal(y, oracle.hash_full(b.n, b.m, s, k)), (path, b.n, b.m)
    assert reps[0]["graph_replayed"] == 0 and reps[1]["graph_replayed"] == 1
    assert sum(reps[0]["blocks_per_path"].values()) == len(bl)
    if path != "auto":
        assert set(paths) == {path}


def test_spectra_slot_reuse():
    # Few slots force pass 1 of later tiles to wait for earlier tiles' pass 3.
    shapes = [(1_000_000 + 7 * i, 300_000 + 11 * i) for i in range(10)]
    bl, keys, seeds = _blocks(shapes, salt=50)
    outs, _, _ = _run_batch(bl, keys, seeds, binding.make_opts(path="ntt31", max_slots=4), runs=3)
    for b, k, s, y in zip(bl, keys, seeds, outs):
        assert np.array_equal(y, oracle.hash_full(b.n, b.m, s, k))


def test_alone_equals_in_the_mix():
    import torch
    bl, keys, seeds = _blocks(MIXED, salt=7)
    outs, _, _ = _run_batch(bl, keys, seeds)
    for b, k, s, y in zip(bl, keys, seeds, outs):
        plan = pkg.Plan(b.n, b.m)
        o = torch.zeros((b.m + 63) // 64, dtype=torch.int64, device="cuda")
        plan.hash(dev(s), dev(k), o)
        torch.cuda.synchronize()
        plan.close()
        assert np.array_equal(host(o), y)


def test_one_shot_and_host_entry():
    import torch
    bl, keys, seeds = _blocks(MIXED[:6], salt=3)
    kd = [dev(k) for k in keys]
    sd = [dev(s) for s in seeds]
    od = [torch.zeros((b.m + 63) // 64, dtype=torch.int64, device="cuda") for b in bl]
    desc = [(b.n, b.m, s, k, o) for b, s, k, o in zip(bl, sd, kd, od)]
    pkg.pa_hash_batched(desc)
    rep = pkg.pa_hash_batched(desc, report=True)
    assert rep["graph_replayed"] == 1
    want = [oracle.hash_full(b.n, b.m, s, k) for b, k, s in zip(bl, keys, seeds)]
    for o, w in zip(od, want):
        assert np.array_equal(host(o), w)
    batch = pkg.pa_batch_plan(desc)
    hout = [np.zeros((b.m + 63) // 64, np.uint64) for b in bl]
    hdesc = [(b.n, b.m, np.ascontiguousarray(s), np.ascontiguousarray(k), o)
             for b, s, k, o in zip(bl, seeds, keys, hout)]
    pkg.pa_batch_run_host(batch, hdesc)
    pkg.pa_batch_destroy(batch)
    for o, w in zip(hout, want):
        assert np.array_equal(o, w)


def test_host_entry_pinned_buffers():
    # Page-locked host buffers take the gather/scatter kernels; one pageable output
    # buffer sends the whole call down the per-buffer copy path. Both must give the
    # oracle's bits, on repeated calls.
    import torch
    bl, keys, seeds = _blocks(MIXED, salt=5)
    want = [oracle.hash_full(b.n, b.m, s, k) for b, k, s in zip(bl, keys, seeds)]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).pin_memory()
    kh = [pin(k) for k in keys]
    sh = [pin(s) for s in seeds]
    batch = pkg.pa_batch_plan([(b.n, b.m, None, None, None) for b in bl])
    for trial in range(3):
        oh = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64).pin_memory() for b in bl]
        outs = list(oh)
        if trial == 2:
            outs[3] = np.full((bl[3].m + 63) // 64, np.uint64(7))  # pageable
        hdesc = [(b.n, b.m, s, k, o) for b, s, k, o in zip(bl, sh, kh, outs)]
        if trial == 1:
            hdesc = pkg.BlockList(hdesc)  # marshalled once, same result
        pkg.pa_batch_run_host(batch, hdesc)
        for i, (o, w) in enumerate(zip(outs, want)):
            got = o if isinstance(o, np.ndarray) else o.numpy().view(np.uint64)
            assert np.array_equal(got, w), (trial, i)
    pkg.pa_batch_destroy(batch)


def test_host_async_two_batches_pipelined():
    # pa_batch_run_host_async: two batches of the same plan alternate on two streams, each
    # call copying keys and seeds in and outputs out by the copy engines without waiting;
    # with different keys per step every output must be the oracle's for its own step's
    # inputs (one pageable output buffer in one step takes the synchronous staging), and the
    # reports read afterwards carry status 0.
    import torch
    shapes = MIXED[:8]
    steps = []
    for salt in (11, 13, 17, 19):
        bl, keys, seeds = _blocks(shapes, salt=salt)
        steps.append((bl, keys, seeds, [oracle.hash_full(b.n, b.m, s, k) for b, k, s in zip(bl, keys, seeds)]))
    bl0 = steps[0][0]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).pin_memory()
    batches = [pkg.pa_batch_plan([(b.n, b.m, None, None, None) for b in bl0]) for _ in range(2)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    held, outs = [], []
    for t, (bl, keys, seeds, _) in enumerate(steps):
        kh, sh = [pin(k) for k in keys], [pin(s) for s in seeds]
        oh = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64).pin_memory() for b in bl]
        if t == 3:
            oh[2] = np.full((bl[2].m + 63) // 64, np.uint64(5))  # pageable
        held.append((kh, sh))  # the host buffers must outlive the enqueued copies
        outs.append(oh)
        pkg.pa_batch_run_host_async(batches[t % 2], [(b.n, b.m, s, k, o) for b, s, k, o in zip(bl, sh, kh, oh)],
                                    streams[t % 2])
    for b, st in zip(batches, streams):
        rep = pkg.pa_batch_get_report(b, st)  # raises PAError on a nonzero device status
        assert sum(rep["blocks_per_path"].values()) == len(shapes)
    for t, (_, _, _, want) in enumerate(steps):
        for i, (o, w) in enumerate(zip(outs[t], want)):
            got = o if isinstance(o, np.ndarray) else o.numpy().view(np.uint64)
            assert np.array_equal(got, w), (t, i)
    for b in batches:
        pkg.pa_batch_destroy(b)


def test_batched_workload_256_blocks():
    import torch
    with open(os.path.join(HERE, "golden", "batched256.json")) as f:
        gold = json.load(f)["blocks"]
    bl = inputs.batched_blocks()
    keys = [b.key() for b in bl]
    seeds = [b.seed() for b in bl]
    outs, reps, paths = _run_batch(bl, keys, seeds)
    for i, (b, y, g) in enumerate(zip(bl, outs, gold)):
        assert (b.n, b.m) == (g["n"], g["m"])
        assert hashlib.sha256(y.astype("<u8").tobytes()).hexdigest() == g["sha256"], i
    # and sampled rows straight from the oracle
    rng = np.random.default_rng(1)
    for i in rng.choice(len(bl), 8, replace=False):
        b = bl[i]
        rows = rng.integers(0, b.m, 64)
        assert np.array_equal(oracle.hash_rows(b.n, b.m, seeds[i], keys[i], rows),
                              oracle.unpack(outs[i], b.m)[rows])


def test_batch_with_segmented_blocks():
    # Blocks whose transform-domain sums run in segments are carried by a batch as their own
    # launch sequences over their own workspaces (captured in the batch's graph with the
    # rest): two forced segmented geometries (8 key x 3 output tiles of 2^18 at N = 2^19,
    # key segments of 3, output slices of 2), compared in full, on the first run and on the
    # graph replay; the plan descriptors report the segments.
    bl, keys, seeds = _blocks([(2_000_007, 600_003), (1_900_001, 700_001)], salt=40)
    opts = binding.make_opts(path="ntt31", log2_transform=19, tile_in=1 << 18,
                             tile_out=1 << 18, fd_mode=2, seg_in=3, seg_out=2)
    import torch
    kd = [dev(k) for k in keys]
    sd = [dev(s) for s in seeds]
    od = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in bl]
    desc = [(b.n, b.m, s, k, o) for b, s, k, o in zip(bl, sd, kd, od)]
    batch = pkg.pa_batch_plan(desc, opts)
    try:
        d = pkg.pa_batch_describe(batch, len(bl))
        assert all(x["segments"] == 6 and x["fd"] == 1 for x in d), d
        for run in range(2):
            rep = pkg.pa_batch_run(batch, desc, report=True)
            assert rep["graph_replayed"] == run
            for b, k, s, o in zip(bl, keys, seeds, od):
                assert np.array_equal(host(o), oracle.hash_full(b.n, b.m, s, k)), (run, b.n, b.m)
            for o in od:
                o.fill_(-1)
    finally:
        pkg.pa_batch_destroy(batch)
