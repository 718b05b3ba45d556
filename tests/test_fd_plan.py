"""Planner of the transform-domain accumulation (host only, no GPU).

Under accumulation the NTT path computes one spectrum per distinct seed-window offset
d = I*M - J*L (Sec. 3 tiling: output tile I, key tile J). The planner's count of those
offsets is checked against brute-force enumeration for every structure it special-cases
(L = M, L a multiple of M, M a multiple of L, neither).
"""
import pytest

import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding

# (n, m, log2 N, L, M)
GEOMS = [(50_003, 20_011, 13, 4096, 4096), (50_003, 20_011, 13, 4096, 2048),
         (30_001, 40_003, 13, 2048, 4096), (40_000, 30_000, 13, 3008, 1088),
         (8_191, 8_193, 13, 4096, 4096), (131_075, 70_001, 14, 8192, 8192),
         (200_000, 3_000, 13, 4096, 1024), (9_000, 200_000, 13, 1024, 4096)]


# one output tile, several key tiles: streamed accumulation (n, m, log2 N, L, M)
STREAMED = [(50_003, 3_000, 13, 4096, 3008), (131_075, 5_000, 14, 8192, 5056),
            (8_191, 1, 13, 4096, 64), (1_000_003, 60_000, 17, 70_016, 60_032)]


def brute_windows(n, m, L, M):
    P, Q = -(-m // M), -(-n // L)
    return len({i * M - j * L for i in range(P) for j in range(Q)})


@pytest.fixture(scope="module")
def lib():
    from paper_1805_02372_gb300 import build
    build.build()
    return binding.load()


@pytest.mark.parametrize("path", ["ntt31", "ntt64"])
@pytest.mark.parametrize("n,m,k,L,M", GEOMS)
def test_window_count_matches_enumeration(lib, path, n, m, k, L, M):
    d = pkg.pa_plan_query(n, m, binding.make_opts(path=path, log2_transform=k, tile_in=L,
                                                  tile_out=M, fd_mode=2))
    assert (d["log2_transform"], d["tile_in"], d["tile_out"]) == (k, L, M)
    assert d["fd"] == 1
    assert d["windows"] == brute_windows(n, m, L, M)
    assert d["kernels_per_call"] == 2


@pytest.mark.parametrize("n,m,k,L,M", GEOMS[:3])
def test_fd_never_when_asked(lib, n, m, k, L, M):
    d = pkg.pa_plan_query(n, m, binding.make_opts(path="ntt31", log2_transform=k, tile_in=L,
                                                  tile_out=M, fd_mode=1))
    assert d["fd"] == 0 and d["windows"] == 0


def test_fd_needs_two_pass_transforms_and_several_pairs(lib):
    # N <= 2^12 runs whole pairs in one CTA: no accumulation.
    d = pkg.pa_plan_query(50_000, 20_000, binding.make_opts(path="ntt31", log2_transform=12,
                                                            tile_in=2048, tile_out=2048,
                                                            fd_mode=2))
    assert d["fd"] == 0
    # a single tile pair has nothing to accumulate
    d = pkg.pa_plan_query(3_000, 1_000, binding.make_opts(path="ntt31", log2_transform=13,
                                                          fd_mode=2))
    assert d["tiles_in"] * d["tiles_out"] == 1 and d["fd"] == 0


def test_fd_mode_validated(lib):
    with pytest.raises(pkg.PAError) as e:
        pkg.pa_plan_query(50_000, 20_000, binding.make_opts(path="ntt31", fd_mode=3))
    assert e.value.status == binding.PA_ERR_INVALID


def test_finite_size_plan_accumulates(lib):
    # n = 1e8, m = 1e7: many output and key tiles, so the planner accumulates, with
    # L = M (P + Q - 1 windows) and far fewer transforms than 3 P Q.
    d = pkg.pa_plan_query(100_000_007, 10_000_000, binding.make_opts(path="ntt31"))
    P, Q = d["tiles_out"], d["tiles_in"]
    assert d["fd"] == 1 and P * Q > 1
    assert d["windows"] == brute_windows(100_000_007, 10_000_000, d["tile_in"], d["tile_out"])
    assert Q + d["windows"] + P < 3 * P * Q / 2


def test_prime_choice(lib):
    q = pkg.pa_plan_query
    # default: 5 * 2^25 + 1 for keys below it (no coefficient counts more than n products),
    # 7 * 2^26 + 1 above, with the same geometry either way
    p28 = 167_772_161
    assert q(1_000_000, 5_000, binding.make_opts(path="ntt31"))["prime_bits"] == 28
    for n, m in ((1_000_000, 5_000), (p28 - 1, 16_000_000), (100_000_007, 10_000_000)):
        d0 = q(n, m, binding.make_opts(path="ntt31"))
        d29 = q(n, m, binding.make_opts(path="ntt31", ntt_prime=29))
        assert d0["prime_bits"] == 28 and d29["prime_bits"] == 29
        for key in ("log2_transform", "tile_in", "tile_out", "fd", "windows", "sum_groups"):
            assert d0[key] == d29[key], key
    assert q(p28, 5_000, binding.make_opts(path="ntt31"))["prime_bits"] == 29
    assert q(1_000_000, 5_000, binding.make_opts(path="ntt31", ntt_prime=28))["prime_bits"] == 28
    assert q(1_000_000, 5_000, binding.make_opts(path="ntt31", ntt_prime=29))["prime_bits"] == 29
    assert q(1_000_000, 5_000, binding.make_opts(path="ntt31", ntt_prime=31))["prime_bits"] == 31
    assert q(1_000_000, 5_000, binding.make_opts(path="ntt64"))["prime_bits"] == 64
    # 7 * 2^26 + 1 = 469,762,049 serves any n: tile pairs count at most L < p products,
    # transform-domain sums at most (p - 1) // L key tiles' worth
    for n in (469_762_048, 469_762_049, 2_013_265_921):
        for prime in (0, 29):
            d = q(n, 5_000, binding.make_opts(path="ntt31", ntt_prime=prime))
            assert d["prime_bits"] == 29
            if d["fd"] == 1:
                assert d["sum_groups"] == -(-d["tiles_in"] // ((469_762_048) // d["tile_in"]))
            elif d["fd"] == 2:
                assert d["tiles_in"] * d["tile_in"] <= 469_762_048 + d["tile_in"]
    # forced 28-bit prime on a longer key: sums of at most (p - 1) // L key tiles
    d = q(1_000_000_007, 100_000_000, binding.make_opts(path="ntt31", ntt_prime=28))
    assert d["prime_bits"] == 28 and d["fd"] == 1
    assert d["sum_groups"] == -(-d["tiles_in"] // ((p28 - 1) // d["tile_in"]))
    for bad in (7, 30):
        with pytest.raises(pkg.PAError):
            q(1_000, 5, binding.make_opts(path="ntt31", ntt_prime=bad))
    assert q(1_000, 5, binding.make_opts(path="direct"))["prime_bits"] == 0


@pytest.mark.parametrize("path,prime", [("ntt31", 28), ("ntt31", 29), ("ntt31", 31), ("ntt64", 0)])
def test_sum_groups(lib, path, prime):
    # pa_opts.fd_group caps the key tiles per transform-domain sum: ceil(Q / g) sums per
    # output tile, each with its own output spectrum
    n, m, k, L, M = GEOMS[0]
    base = pkg.pa_plan_query(n, m, binding.make_opts(path=path, log2_transform=k, tile_in=L,
                                                     tile_out=M, fd_mode=2, ntt_prime=prime))
    assert base["fd"] == 1 and base["sum_groups"] == 1
    Q, P = base["tiles_in"], base["tiles_out"]
    elem = 8 if path == "ntt64" else 4
    for g in (1, 2, 4, Q - 1, Q, Q + 5):
        d = pkg.pa_plan_query(n, m, binding.make_opts(path=path, log2_transform=k, tile_in=L,
                                                      tile_out=M, fd_mode=2, ntt_prime=prime,
                                                      fd_group=g))
        G = -(-Q // min(g, Q))
        assert d["fd"] == 1 and d["sum_groups"] == G
        assert d["workspace_bytes"] - base["workspace_bytes"] >= (G - 1) * P * elem << k


@pytest.mark.parametrize("path", ["ntt31", "ntt64"])
@pytest.mark.parametrize("n,m,k,L,M", STREAMED)
def test_streamed_plan(lib, path, n, m, k, L, M):
    d = pkg.pa_plan_query(n, m, binding.make_opts(path=path, log2_transform=k, tile_in=L,
                                                  tile_out=M, fd_mode=2))
    assert d["tiles_out"] == 1 and d["tiles_in"] == -(-n // L) > 1
    assert d["fd"] == 2 and d["windows"] == d["tiles_in"] == brute_windows(n, m, L, M)


def test_streamed_chosen_for_batched_shapes(lib):
    # n = 4e6, m = 2e6 at N = 2^22 is two key tiles and one output tile: the model
    # prices 2Q + 1 transforms below 3Q
    d = pkg.pa_plan_query(4_000_000, 2_000_000, binding.make_opts(path="ntt31"))
    assert d["tiles_out"] == 1 and d["tiles_in"] >= 2 and d["fd"] == 2


def test_largest_transform_only_under_multi_output_accumulation(lib):
    # 2^23-point transforms (pass-2 rows of 2^12 points) run only through the multi-output
    # sums, a single output tile included (one output per sum item); standard pairs and
    # the streamed body stop at 2^22, and nothing goes above 2^23.
    q = pkg.pa_plan_query
    n, m, L, M = 20_000_003, 9_000_000, 1 << 22, 1 << 22
    for path in ("ntt31", "ntt64"):
        d = q(n, m, binding.make_opts(path=path, log2_transform=23, tile_in=L, tile_out=M))
        assert (d["log2_transform"], d["fd"]) == (23, 1)
        assert d["windows"] == brute_windows(n, m, L, M)
        # one output tile: the sums with a single output (W = Q windows), not streamed
        d = q(n, 4_000_000, binding.make_opts(path=path, log2_transform=23, tile_in=L,
                                              tile_out=L, fd_mode=2))
        assert (d["log2_transform"], d["fd"], d["tiles_out"]) == (23, 1, 1)
        assert d["windows"] == d["tiles_in"] == brute_windows(n, 4_000_000, L, L)
    for args in ((n, m, dict(fd_mode=1, tile_in=L, tile_out=M)),   # standard pairs
                 (3_000, 1_000, dict())):                           # a single pair
        with pytest.raises(pkg.PAError) as e:
            q(args[0], args[1], binding.make_opts(path="ntt31", log2_transform=23, **args[2]))
        assert e.value.status == binding.PA_ERR_UNSUPPORTED
    with pytest.raises(pkg.PAError):
        q(n, m, binding.make_opts(path="ntt31", log2_transform=24))


def test_finite_and_paper_scale_take_the_largest_transform(lib):
    # The summed products of accumulation number P Q N, about 4 m n / N: at n = 1e8 and
    # 1e9 (l = 10%) the model prefers 2^23 points to 2^22.
    for n, m in ((100_000_007, 10_000_000), (1_000_000_007, 100_000_000)):
        d = pkg.pa_plan_query(n, m, binding.make_opts(path="ntt31"))
        assert (d["log2_transform"], d["fd"]) == (23, 1)
        assert d["tile_in"] + d["tile_out"] <= 1 << 23


@pytest.mark.parametrize("n,m,k,L,M", STREAMED[:3])
def test_several_sums_never_stream(lib, n, m, k, L, M):
    # The streamed body keeps one accumulator over every key tile, so a block whose key
    # needs several sums (here forced by fd_group) takes the multi-output sums with a
    # single output tile instead.
    opts = dict(path="ntt31", log2_transform=k, tile_in=L, tile_out=M, fd_mode=2)
    d = pkg.pa_plan_query(n, m, binding.make_opts(**opts))
    assert d["fd"] == 2 and d["sum_groups"] == 1
    g = pkg.pa_plan_query(n, m, binding.make_opts(fd_group=1, **opts))
    assert (g["fd"], g["tiles_out"], g["sum_groups"]) == (1, 1, g["tiles_in"])
    assert g["windows"] == g["tiles_in"]



def test_segmented_plan_beyond_the_resident_cap(lib):
    # n = 1e10, l = 10%: resident spectra would need about 330 GB; the plan segments the
    # key tiles (one sum's worth per segment) within the default 32 GiB of spectra
    n, m = 10_000_000_019, 1_000_000_000
    d = pkg.pa_plan_query(n, m, binding.make_opts(path="ntt31"))
    assert d["fd"] == 1 and d["prime_bits"] == 29 and d["segments"] > 1
    P, Q = d["tiles_out"], d["tiles_in"]
    assert d["segments"] == -(-P // d["seg_out"]) * -(-Q // d["seg_in"])
    assert d["workspace_bytes"] < (33 << 30)
    # a segment's sums stay below the 29-bit prime: at most (p - 1) / L key tiles per sum
    assert d["seg_in"] * d["tile_in"] <= 469762049 - 1 or d["sum_groups"] > d["segments"]
    assert d["kernels_per_call"] == d["segments"] + 1


def test_segment_cap_shrinks_the_segments(lib):
    n, m = 10_000_000_019, 1_000_000_000
    big = pkg.pa_plan_query(n, m, binding.make_opts(path="ntt31"))
    small = pkg.pa_plan_query(n, m, binding.make_opts(path="ntt31", seg_cap_gib=8))
    # the cap bounds a segment's spectra; every segment's work-list tables come on top
    assert small["workspace_bytes"] < min(big["workspace_bytes"], 12 << 30)
    assert small["segments"] > big["segments"]


def test_forced_segments_shape(lib):
    d = pkg.pa_plan_query(2_000_007, 600_003, binding.make_opts(
        path="ntt31", log2_transform=19, tile_in=1 << 18, tile_out=1 << 18, fd_mode=2,
        seg_in=3, seg_out=2))
    assert (d["tiles_in"], d["tiles_out"], d["seg_in"], d["seg_out"]) == (8, 3, 3, 2)
    assert d["segments"] == 2 * 3 and d["sum_groups"] == 3


def test_planning_stays_fast_for_serving_sizes(lib):
    # the geometry search must not enumerate window offsets for implausible candidates (a
    # wave of the server plans its blocks on the latency path): keys up to 1e8 bits plan
    # in well under a tenth of a second on the host
    import time
    shapes = [(79_938_100, 13_501_589), (96_422_116, 11_557_350), (97_228_129, 42_449_279),
              (27_259_615, 10_707_482)]
    t0 = time.perf_counter()
    for n, m in shapes:
        pkg.pa_plan_query(n, m, binding.make_opts(path="ntt31"))
    assert (time.perf_counter() - t0) / len(shapes) < 0.05


@pytest.mark.parametrize("path", ["ntt31", "ntt64"])
def test_oversized_standard_plans_refused_before_layout(lib, path):
    # Without transform-domain sums a key of 1e10 bits needs about 2.3e6 tile pairs of 2^22
    # points, each a tile record and 1280 (32-bit primes) or 2560 (64-bit prime) work items:
    # billions of list entries. The planner refuses such a plan with PA_ERR_UNSUPPORTED at
    # once instead of building the list (which took 40 s and 28 GB of host memory for the
    # 29-bit prime, and threw std::bad_alloc through the C interface for the 64-bit one).
    # Tiny forced tiles on a long key are refused the same way.
    import time
    cases = [(10_000_000_019, 1_000_000_000, dict(fd_mode=1)),
             (10_000_000_019, 1_000_000_000, dict(outer_mode=1, seg_in=3, seg_out=2)),
             (100_000_007, 10_000_000, dict(log2_transform=13, tile_in=4096, tile_out=4096,
                                            fd_mode=1))]
    for n, m, extra in cases:
        t0 = time.perf_counter()
        with pytest.raises(pkg.PAError) as e:
            pkg.pa_plan_query(n, m, binding.make_opts(path=path, **extra))
        assert e.value.status == binding.PA_ERR_UNSUPPORTED
        assert time.perf_counter() - t0 < 2.0
    # the largest standard plan still accepted: 1e9 bits with sums forbidden
    d = pkg.pa_plan_query(1_000_000_007, 100_000_000, binding.make_opts(path=path, fd_mode=1))
    assert d["fd"] == 0 and d["tiles_in"] * d["tiles_out"] > 1000


def test_outer_convolutions_chosen_and_forced(lib):
    # forced on a small equal-tile geometry, refused when asked never; the model takes them
    # for long keys (many output and key tiles) and not for the finite-size block (3 x 24)
    geo = dict(log2_transform=15, tile_in=1 << 14, tile_out=1 << 14, fd_mode=2)
    d = pkg.pa_plan_query(2_000_007, 600_003, binding.make_opts(path="ntt31", outer_mode=2, **geo))
    assert d["outer_log2"] == 8 and d["outer_slice"] == 37  # 37 + 123 - 1 = 159 -> 256 points
    d = pkg.pa_plan_query(2_000_007, 600_003, binding.make_opts(path="ntt31", outer_mode=1, **geo))
    assert d["outer_log2"] == 0
    big = pkg.pa_plan_query(10_000_000_019, 1_000_000_000, binding.make_opts(path="ntt31"))
    assert big["outer_log2"] > 0 and big["segments"] > 1
    # measured: outer sums 26% faster at n = 3e9 (72 output tiles), 28% slower at n = 1e9 (24)
    mid = pkg.pa_plan_query(3_000_000_019, 300_000_000, binding.make_opts(path="ntt31"))
    assert mid["outer_log2"] > 0 and mid["segments"] == 0
    low = pkg.pa_plan_query(1_000_000_007, 100_000_000, binding.make_opts(path="ntt31"))
    assert low["outer_log2"] == 0
    fs = pkg.pa_plan_query(100_000_007, 10_000_000, binding.make_opts(path="ntt31"))
    assert fs["outer_log2"] == 0
    with pytest.raises(pkg.PAError):
        pkg.pa_plan_query(2_000_007, 600_003, binding.make_opts(path="ntt31", outer_mode=3))
