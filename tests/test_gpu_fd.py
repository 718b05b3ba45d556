"""Transform-domain accumulation on the GPU: bit-exact against the oracle.

Every window-offset structure the planner distinguishes (L = M, L = 2M, M = 2L, neither
dividing the other), both prime fields, ragged tails, fd blocks next to standard tiles
in one persistent launch, the largest (2^23-point) transforms, and the finite-size
workload (n = 1e8, m = 1e7) on sampled rows plus linearity.
"""
import numpy as np
import pytest

import oracle
import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding, inputs
from gpu_util import dev, host, run_path

pytestmark = pytest.mark.gpu

# (n, m, log2 N, L, M)
GEOMS = [(50_003, 20_011, 13, 4096, 4096), (50_003, 20_011, 13, 4096, 2048),
         (30_001, 40_003, 13, 2048, 4096), (40_000, 30_000, 13, 3008, 1088),
         (8_191, 8_193, 13, 4096, 4096), (131_075, 70_001, 14, 8192, 8192),
         (200_000, 3_000, 13, 4096, 1024), (9_000, 200_000, 13, 1024, 4096)]


@pytest.mark.parametrize("path,prime", [("ntt31", 28), ("ntt31", 29), ("ntt31", 31), ("ntt64", 0)])
@pytest.mark.parametrize("n,m,k,L,M", GEOMS)
def test_fd_matches_oracle(path, prime, n, m, k, L, M):
    blk = inputs.single_block(n, m, 31 + n, 37 + m)
    key, seed = blk.key(), blk.seed()
    want = oracle.hash_full(n, m, seed, key)
    got, desc = run_path(n, m, key, seed, path=path, log2_transform=k, tile_in=L, tile_out=M,
                         fd_mode=2, ntt_prime=prime)
    assert desc["fd"] == 1 and desc["prime_bits"] == (prime or 64)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{path} {desc}: {bad.size} words differ, first at {bad[0]}"


# one output tile, several key tiles: streamed accumulation (n, m, log2 N, L, M)
STREAMED = [(50_003, 3_000, 13, 4096, 3008), (131_075, 5_000, 14, 8192, 5056),
            (8_191, 1, 13, 4096, 64), (1_000_003, 60_000, 17, 70_016, 60_032)]


@pytest.mark.parametrize("path,prime", [("ntt31", 28), ("ntt31", 29), ("ntt31", 31), ("ntt64", 0)])
@pytest.mark.parametrize("n,m,k,L,M", STREAMED)
def test_streamed_matches_oracle(path, prime, n, m, k, L, M):
    blk = inputs.single_block(n, m, 41 + n, 43 + m)
    key, seed = blk.key(), blk.seed()
    want = oracle.hash_full(n, m, seed, key)
    got, desc = run_path(n, m, key, seed, path=path, log2_transform=k, tile_in=L, tile_out=M,
                         fd_mode=2, ntt_prime=prime)
    assert desc["fd"] == 2 and desc["tiles_out"] == 1
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{path} {desc}: {bad.size} words differ, first at {bad[0]}"


@pytest.mark.parametrize("kind", ["ones", "seed_ones"])
def test_fd_largest_coefficients(kind):
    # all-ones inputs give the largest sums (every coefficient counts L products per key
    # tile, up to n in one transform-domain sum)
    n, m = 60_001, 25_003
    key = np.full((n + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    seed = np.full((n + m - 1 + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    if kind == "seed_ones":
        key = inputs.random_bits(n, 5)
    want = oracle.hash_full(n, m, seed, key)
    got, desc = run_path(n, m, key, seed, path="ntt31", log2_transform=13, tile_in=4096,
                         tile_out=4096, fd_mode=2)
    assert desc["fd"] == 1 and np.array_equal(got, want)


@pytest.mark.parametrize("path,prime", [("ntt31", 28), ("ntt31", 29), ("ntt31", 31), ("ntt64", 0)])
@pytest.mark.parametrize("geom", [GEOMS[0], GEOMS[3], GEOMS[5], GEOMS[7]])
@pytest.mark.parametrize("group", [1, 3])
def test_grouped_sums_match_oracle(path, prime, geom, group):
    # Several transform-domain sums per output tile (pa_opts.fd_group key tiles each), each
    # with its own inverse transform, their output bits XOR-merged (Eq. finalkey): sliding
    # (L = M) and looked-up windows, ragged last groups.
    n, m, k, L, M = geom
    blk = inputs.single_block(n, m, 61 + n, 67 + m)
    key, seed = blk.key(), blk.seed()
    want = oracle.hash_full(n, m, seed, key)
    got, desc = run_path(n, m, key, seed, path=path, log2_transform=k, tile_in=L, tile_out=M,
                         fd_mode=2, ntt_prime=prime, fd_group=group)
    assert desc["fd"] == 1 and desc["sum_groups"] == -(-desc["tiles_in"] // group) > 1
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{path} {desc}: {bad.size} words differ, first at {bad[0]}"


def test_grouped_sums_at_the_exactness_limit():
    # All-ones key and seed: every coefficient of a sum over g key tiles counts g L
    # products. With L = 2^23 - 4096 the 29-bit prime p = 469,762,049 allows g = 56
    # (56 L = 469,532,672 < p; 57 L would wrap), so n = 5e8 + 1 takes two sums (56 + 4 key
    # tiles) per output tile. Every output bit is n mod 2 (each row of T is all ones).
    n, m = 500_000_001, 3_001
    L, M = (1 << 23) - 4096, 4096
    key = np.full((n + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    seed = np.full((n + m - 1 + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    got, desc = run_path(n, m, key, seed, path="ntt31", log2_transform=23, tile_in=L, tile_out=M,
                         fd_mode=2)
    assert (desc["prime_bits"], desc["fd"], desc["tiles_in"], desc["sum_groups"]) == (29, 1, 60, 2)
    assert ((469_762_049 - 1) // L, 56 * L < 469_762_049 <= 57 * L) == (56, True)
    bits = oracle.unpack(got, m)
    assert np.all(bits == (n & 1))
    if m % 64:
        assert int(got[-1]) >> (m % 64) == 0
    rows = np.array([0, 1, m // 2, m - 1])
    assert np.array_equal(bits[rows], oracle.hash_rows(n, m, seed, key, rows))


def test_grouped_sums_at_the_exactness_limit_28bit():
    # The same at the 28-bit prime p = 167,772,161 (forced): with L = 2^23 - 4096 a sum
    # covers g = 20 key tiles (20 L = 167,690,240 < p; 21 L would wrap), so n = 2e8 + 1
    # takes two sums (20 + 4 key tiles) per output tile and the first sum's coefficients
    # reach 20 L, within 82,000 of p: the lazily reduced rounds run on counts next to the
    # prime. Every output bit is n mod 2.
    n, m = 200_000_001, 3_001
    L, M = (1 << 23) - 4096, 4096
    key = np.full((n + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    seed = np.full((n + m - 1 + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    got, desc = run_path(n, m, key, seed, path="ntt31", log2_transform=23, tile_in=L, tile_out=M,
                         fd_mode=2, ntt_prime=28)
    assert (desc["prime_bits"], desc["fd"], desc["tiles_in"], desc["sum_groups"]) == (28, 1, 24, 2)
    assert ((167_772_161 - 1) // L, 20 * L < 167_772_161 <= 21 * L) == (20, True)
    bits = oracle.unpack(got, m)
    assert np.all(bits == (n & 1))


def test_fd_and_standard_tiles_in_one_launch():
    import torch
    shapes = [(50_003, 20_011), (3_001, 1_000), (20_000, 9_000), (1, 1), (70_001, 64),
              (8_191, 8_193), (60_007, 3_001), (40_001, 100)]
    bl = [inputs.single_block(n, m, 500 + 2 * i, 501 + 2 * i) for i, (n, m) in enumerate(shapes)]
    keys, seeds = [b.key() for b in bl], [b.seed() for b in bl]
    kd, sd = [dev(k) for k in keys], [dev(s) for s in seeds]
    od = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in bl]
    desc = [(b.n, b.m, s, k, o) for b, s, k, o in zip(bl, sd, kd, od)]
    opts = binding.make_opts(path="ntt31", log2_transform=13, tile_in=4096, tile_out=4096,
                             fd_mode=2)
    batch = pkg.pa_batch_plan(desc, opts)
    try:
        plans = pkg.pa_batch_describe(batch, len(bl))
        assert {d["fd"] for d in plans} == {0, 1, 2}
        for run in range(3):  # first run captures the graph, later runs replay it
            for o in od:
                o.fill_(-1)
            rep = pkg.pa_batch_run(batch, desc, report=True)
            assert rep["graph_replayed"] == (1 if run else 0)
            for b, k, s, o in zip(bl, keys, seeds, od):
                assert np.array_equal(host(o), oracle.hash_full(b.n, b.m, s, k)), (run, b.n, b.m)
    finally:
        pkg.pa_batch_destroy(batch)


def test_fd_equals_standard_at_size():
    # n = 4e6, m = 1.5e6 at N = 2^21, L = M = 2^20: 6 output x 4 key tiles
    n, m = 4_000_003, 1_500_001
    blk = inputs.single_block(n, m, 71, 73)
    key, seed = blk.key(), blk.seed()
    a, da = run_path(n, m, key, seed, path="ntt31", log2_transform=21, tile_in=1 << 20,
                     tile_out=1 << 20, fd_mode=2)
    b, db = run_path(n, m, key, seed, path="ntt31", log2_transform=21, tile_in=1 << 20,
                     tile_out=1 << 20, fd_mode=1)
    assert da["fd"] == 1 and db["fd"] == 0
    assert np.array_equal(a, b)
    rows = np.unique(np.concatenate([np.random.default_rng(3).integers(0, m, 2000),
                                     [0, m - 1, (1 << 20) - 1, 1 << 20]]))
    assert np.array_equal(oracle.unpack(a, m)[rows], oracle.hash_rows(n, m, seed, key, rows))


# 2^23-point transforms (the largest, multi-output accumulation only): pass-1 columns of
# 2^11 points and pass-2 rows of 2^12, summed in two 2048-element chunks per row.
# L = 15 * 2^19, M = 2^19: 2 x 2 tiles whose windows are looked up (L != M);
# L = 7 * 2^20, M = 2^20: one output tile, the sums with a single output per item.
BIG = (8_000_003, 600_001, 23)
BIG_TILES = [(15 << 19, 1 << 19, 2), (7 << 20, 1 << 20, 1)]
# the same at one key tile per sum: two sums per output tile


@pytest.fixture(scope="module")
def big_case():
    n, m = BIG[:2]
    blk = inputs.single_block(n, m, 81, 83)
    key, seed = blk.key(), blk.seed()
    return key, seed, oracle.hash_full(n, m, seed, key)


@pytest.mark.parametrize("group", [0, 1])
@pytest.mark.parametrize("L,M,P", BIG_TILES)
@pytest.mark.parametrize("path,prime", [("ntt31", 28), ("ntt31", 29), ("ntt31", 31), ("ntt64", 0)])
def test_largest_transform_matches_oracle(big_case, path, prime, L, M, P, group):
    n, m, k = BIG
    key, seed, want = big_case
    got, desc = run_path(n, m, key, seed, path=path, log2_transform=k, tile_in=L, tile_out=M,
                         fd_mode=2, ntt_prime=prime, fd_group=group)
    assert (desc["log2_transform"], desc["fd"], desc["tiles_in"], desc["tiles_out"]) == (23, 1, 2, P)
    assert desc["sum_groups"] == (2 if group == 1 else 1)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, f"{path} {desc}: {bad.size} words differ, first at {bad[0]}"


def test_largest_transform_sliding_windows_sampled_rows():
    # L = M = 2^22: 3 output x 3 key tiles, windows d0 + I - J (the sliding sum)
    n, m = 10_000_019, 9_000_011
    blk = inputs.single_block(n, m, 85, 87)
    key, seed = blk.key(), blk.seed()
    got, desc = run_path(n, m, key, seed, path="ntt31", log2_transform=23, tile_in=1 << 22,
                         tile_out=1 << 22, fd_mode=2)
    assert (desc["log2_transform"], desc["fd"], desc["tiles_out"]) == (23, 1, 3)
    M = 1 << 22
    edges = [r for i in range(3) for r in (i * M - 1, i * M, i * M + 1, i * M + 2047, i * M + 2048)
             if 0 <= r < m]
    rows = np.unique(np.concatenate([np.random.default_rng(5).integers(0, m, 400), edges, [m - 1]]))
    assert np.array_equal(oracle.unpack(got, m)[rows], oracle.hash_rows(n, m, seed, key, rows))
    if m % 64:
        assert int(got[-1]) >> (m % 64) == 0


def test_largest_transform_in_a_mixed_batch():
    # One autotuned persistent launch holding a 2^23-point accumulated block (64 Mbit,
    # l = 10%) next to streamed, standard and one-CTA blocks: the launch's shared memory is
    # the largest body's, and stage tables of 2^11- and 2^12-point passes alternate in the
    # CTAs' cache. Small blocks against the full oracle, the large one on sampled rows.
    import torch
    shapes = [(64_000_000, 6_400_000), (1_000_003, 60_000), (300_007, 150_001), (3_001, 1_000),
              (2_000_003, 400_001), (70_001, 64)]
    bl = [inputs.single_block(n, m, 701 + i, 801 + i) for i, (n, m) in enumerate(shapes)]
    keys, seeds = [b.key() for b in bl], [b.seed() for b in bl]
    od = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in bl]
    desc = [(b.n, b.m, dev(s), dev(k), o) for b, s, k, o in zip(bl, seeds, keys, od)]
    batch = pkg.pa_batch_plan(desc, binding.make_opts(path="auto"))
    try:
        plans = pkg.pa_batch_describe(batch, len(bl))
        assert (plans[0]["log2_transform"], plans[0]["fd"]) == (23, 1), plans[0]
        assert any(d["path_name"] in ("ntt31", "ntt64") and d["log2_transform"] <= 22 for d in plans[1:])
        b, m, M = bl[0], bl[0].m, plans[0]["tile_out"]
        edges = [r for i in range(plans[0]["tiles_out"]) for r in (i * M - 1, i * M) if 0 <= r < m]
        rows = np.unique(np.concatenate([np.random.default_rng(11).integers(0, m, 150), edges, [m - 1]]))
        want0 = oracle.hash_rows(b.n, m, seeds[0], keys[0], rows)
        want = [oracle.hash_full(b.n, b.m, s, k) for b, k, s in zip(bl[1:], keys[1:], seeds[1:])]
        for run in range(2):  # first run captures the graph, the second replays it
            for o in od:
                o.fill_(-1)
            pkg.pa_batch_run(batch, desc)
            assert np.array_equal(oracle.unpack(host(od[0]), m)[rows], want0), run
            for b, o, w in zip(bl[1:], od[1:], want):
                assert np.array_equal(host(o), w), (run, b.n, b.m)
    finally:
        pkg.pa_batch_destroy(batch)


def test_finite_size_fd_sampled_rows():
    b = inputs.FINITE_SIZE
    key, seed = b.key(), b.seed()
    got, desc = run_path(b.n, b.m, key, seed, path="ntt31")
    assert desc["fd"] == 1
    rng = np.random.default_rng(9)
    M = desc["tile_out"]
    edges = [r for i in range(desc["tiles_out"]) for r in (i * M - 1, i * M, i * M + 1)
             if 0 <= r < b.m]
    rows = np.unique(np.concatenate([rng.integers(0, b.m, 3000), edges, [b.m - 1]]))
    want = oracle.hash_rows(b.n, b.m, seed, key, rows)
    assert np.array_equal(oracle.unpack(got, b.m)[rows], want)
    if b.m % 64:
        assert int(got[-1]) >> (b.m % 64) == 0
    key2 = inputs.random_bits(b.n, 778)
    g2, _ = run_path(b.n, b.m, key2, seed, path="ntt31")
    g12, _ = run_path(b.n, b.m, key ^ key2, seed, path="ntt31")
    assert np.array_equal(g12, got ^ g2)


def test_autotuned_batch_honours_fd_group():
    # pa_opts.fd_group binds the autotuner's NTT blocks in a batch: with one key tile per
    # sum an accumulated block has a sum per key tile, and no block with several key
    # tiles streams (one accumulator over all of them); the bits stay the oracle's.
    import torch
    shapes = [(1_000_003, 60_000), (2_000_003, 400_001), (4_000_037, 40_009), (3_000_017, 1_500_007)]
    bl = [inputs.single_block(n, m, 521 + i, 621 + i) for i, (n, m) in enumerate(shapes)]
    keys, seeds = [b.key() for b in bl], [b.seed() for b in bl]
    want = [oracle.hash_full(b.n, b.m, s, k) for b, k, s in zip(bl, keys, seeds)]
    outs = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in bl]
    desc = [(b.n, b.m, dev(s), dev(k), o) for b, s, k, o in zip(bl, seeds, keys, outs)]
    batch = pkg.pa_batch_plan(desc, binding.make_opts(path="auto", fd_group=1))
    try:
        plans = pkg.pa_batch_describe(batch, len(bl))
        for p in plans:
            if p["fd"] == 1:
                assert p["sum_groups"] == p["tiles_in"], p
            if p["fd"] == 2:
                assert p["tiles_in"] == 1, p
        pkg.pa_batch_run(batch, desc)
        for o, w in zip(outs, want):
            assert np.array_equal(host(o), w)
    finally:
        pkg.pa_batch_destroy(batch)


def test_autotuned_batch_honours_fd_mode():
    # pa_opts.fd_mode applies to the autotuner's NTT blocks in a batch too: 1 plans no
    # transform-domain accumulation, and the bits stay the oracle's either way.
    import torch
    shapes = [(1_000_003, 60_000), (2_000_003, 400_001), (300_007, 150_001), (4_000_037, 40_009)]
    bl = [inputs.single_block(n, m, 501 + i, 601 + i) for i, (n, m) in enumerate(shapes)]
    keys, seeds = [b.key() for b in bl], [b.seed() for b in bl]
    want = [oracle.hash_full(b.n, b.m, s, k) for b, k, s in zip(bl, keys, seeds)]
    for mode in (0, 1):
        outs = [torch.full(((b.m + 63) // 64,), -1, dtype=torch.int64, device="cuda") for b in bl]
        desc = [(b.n, b.m, dev(s), dev(k), o) for b, s, k, o in zip(bl, seeds, keys, outs)]
        batch = pkg.pa_batch_plan(desc, binding.make_opts(path="auto", fd_mode=mode))
        plans = pkg.pa_batch_describe(batch, len(bl))
        pkg.pa_batch_run(batch, desc)
        pkg.pa_batch_destroy(batch)
        if mode == 1:
            assert all(p["fd"] == 0 for p in plans if p["path_name"] in ("ntt31", "ntt64"))
        for o, w in zip(outs, want):
            assert np.array_equal(host(o), w), mode
