"""Bit-exact parity of every CUDA path with the CPU oracle (through the C ABI).

Shapes span several tiles of every path plus ragged tails; the named workloads run
at full size (the 1e8-bit one is checked on sampled rows the oracle evaluates one
by one, plus linearity, which holds at any size).
"""
import functools

import numpy as np
import pytest

import oracle
import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding, inputs
from gpu_util import dev, host, run_path

pytestmark = pytest.mark.gpu

PATHS = ["direct", "ntt64", "ntt31", "fft", "block_int8", "block_fp8"]

SHAPES = [(1, 1), (1, 100), (100, 1), (2, 2), (31, 33), (64, 64), (65, 63), (1000, 1),
          (1, 5000), (4097, 4095), (12345, 777), (70001, 64), (64, 70001), (33333, 33333),
          (262_145, 131_071), (1_048_577, 3)]


@functools.lru_cache(maxsize=None)
def _case(n, m, ks, ss):
    blk = inputs.single_block(n, m, ks, ss)
    key, seed = blk.key(), blk.seed()
    return key, seed, oracle.hash_full(n, m, seed, key)


def _supported(path, n, m):
    try:
        pkg.pa_plan_query(n, m, binding.make_opts(path=path))
        return True
    except pkg.PAError as e:
        if e.status in (binding.PA_ERR_UNSUPPORTED, binding.PA_ERR_PRECISION):
            return False
        raise


def _check(path, n, m, key, seed, want, **opts):
    if not _supported(path, n, m):
        pytest.skip(f"{path} does not take n={n}, m={m}")
    got, desc = run_path(n, m, key, seed, path=path, **opts)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (f"{path} n={n} m={m} plan={desc}: {bad.size} words differ, "
                           f"first at word {bad[0]}")


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("n,m", SHAPES)
def test_shapes(path, n, m):
    key, seed, want = _case(n, m, 11 + n, 13 + m)
    _check(path, n, m, key, seed, want)


@pytest.mark.parametrize("prime", [29, 31])
@pytest.mark.parametrize("n,m", SHAPES)
def test_shapes_other_primes(n, m, prime):
    # the NTT31 path takes the 28-bit prime below its bound; force the 29- and 31-bit ones
    key, seed, want = _case(n, m, 11 + n, 13 + m)
    _check("ntt31", n, m, key, seed, want, ntt_prime=prime)


@pytest.mark.parametrize("path", PATHS)
def test_plain_single_block(path):
    b = inputs.PLAIN_SINGLE
    key, seed, want = _case(b.n, b.m, b.key_stream, b.seed_stream)
    _check(path, b.n, b.m, key, seed, want)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("m", [10_000, 250_000, 500_000])
def test_plain_vs_transform(path, m):
    b = inputs.single_block(1_000_000, m)
    key, seed, want = _case(b.n, b.m, b.key_stream, b.seed_stream)
    _check(path, b.n, b.m, key, seed, want)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("kind", ["ones", "zeros", "key_one_bit", "seed_one_bit"])
def test_structured_inputs(path, kind):
    # All-ones key and seed give the largest integer coefficients (the FP worst case).
    n, m = 200_003, 70_001
    kw, sw = (n + 63) // 64, (n + m - 1 + 63) // 64
    key = np.full(kw, np.uint64(0xFFFFFFFFFFFFFFFF))
    seed = np.full(sw, np.uint64(0xFFFFFFFFFFFFFFFF))
    if kind == "zeros":
        key[:] = 0
    elif kind == "key_one_bit":
        key[:] = 0
        key[1234 // 64] = np.uint64(1) << np.uint64(1234 % 64)
    elif kind == "seed_one_bit":
        seed[:] = 0
        t = n - 1 + 5000
        seed[t // 64] = np.uint64(1) << np.uint64(t % 64)
        key = inputs.random_bits(n, 99)
    want = oracle.hash_full(n, m, seed, key)
    _check(path, n, m, key, seed, want)


@pytest.mark.parametrize("path", PATHS)
def test_finite_size_sampled_rows(path):
    b = inputs.FINITE_SIZE
    if not _supported(path, b.n, b.m):
        pytest.skip(f"{path} does not take the finite-size workload")
    key, seed = b.key(), b.seed()
    got, desc = run_path(b.n, b.m, key, seed, path=path)
    rng = np.random.default_rng(5)
    rows = np.unique(np.concatenate([rng.integers(0, b.m, 3000), [0, 1, 63, 64, b.m - 1],
                                     np.arange(0, b.m, max(1, b.m // 997))]))
    want = oracle.hash_rows(b.n, b.m, seed, key, rows)
    gbits = oracle.unpack(got, b.m)[rows]
    assert np.array_equal(gbits, want), f"{path}: sampled rows differ ({desc})"
    # Output tail bits zero.
    if b.m % 64:
        assert int(got[-1]) >> (b.m % 64) == 0
    if path in ("direct", "block_int8", "fft"):
        return  # 1e15 bit products per run (3-21 s): sampled rows only
    # Linearity in the key holds at any size: h(x1 ^ x2) = h(x1) ^ h(x2).
    key2 = inputs.random_bits(b.n, 777)
    g2, _ = run_path(b.n, b.m, key2, seed, path=path)
    g12, _ = run_path(b.n, b.m, key ^ key2, seed, path=path)
    assert np.array_equal(g12, got ^ g2)


def _golden(name):
    import json
    import os
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)) as f:
        return json.load(f)


def _sha(words):
    import hashlib
    return hashlib.sha256(np.ascontiguousarray(words, dtype="<u8").tobytes()).hexdigest()


@pytest.mark.parametrize("path,opts", [("ntt31", {}), ("ntt31", {"ntt_prime": 29}),
                                       ("ntt31", {"ntt_prime": 31}), ("ntt64", {}),
                                       ("block_fp8", {}), ("direct", {}), ("block_int8", {}),
                                       ("fft", {})])
def test_finite_size_full_output(path, opts):
    # Every output bit of the finite-size block (n = 100,000,007, m = 1e7: 1e15 bit products)
    # against the SHA-256 of the oracle's full output, stored by tests/golden/make_golden.py;
    # the digests of 16 equal slices of the output words name the rows of any mismatch.
    g = _golden("finite_size.json")
    b = inputs.FINITE_SIZE
    assert (g["n"], g["m"]) == (b.n, b.m)
    got, desc = run_path(b.n, b.m, b.key(), b.seed(), path=path, **opts)
    if _sha(got) != g["sha256"]:
        w, k = got.size, g["slices"]
        bad = [i for i in range(k) if _sha(got[i * w // k:(i + 1) * w // k]) != g["slice_sha256"][i]]
        pytest.fail(f"{path} {opts}: output differs from the oracle in word slices {bad} of {k} "
                    f"({desc})")


def test_misaligned_buffers_rejected():
    import torch
    n, m = 1000, 100
    plan = pkg.Plan(n, m, path="direct")
    buf = torch.zeros(64, dtype=torch.int64, device="cuda")
    raw = buf.data_ptr() + 8
    with pytest.raises(pkg.PAError) as e:
        pkg.pa_hash(plan.handle, raw, buf, buf)
    assert e.value.status == binding.PA_ERR_ALIGN
    with pytest.raises(pkg.PAError) as e:
        pkg.pa_hash(plan.handle, 0, buf, buf)
    assert e.value.status == binding.PA_ERR_INVALID
    plan.close()


@pytest.mark.parametrize("path", PATHS)
def test_host_entry_point(path):
    n, m = 100_003, 25_000
    if not _supported(path, n, m):
        pytest.skip("unsupported")
    key, seed, want = _case(n, m, 1, 2)
    plan = pkg.Plan(n, m, path=path)
    out = np.zeros_like(want)
    plan.hash_host(np.ascontiguousarray(seed), np.ascontiguousarray(key), out)
    plan.close()
    assert np.array_equal(out, want)


@pytest.mark.parametrize("b", [128, 256, 512])
@pytest.mark.parametrize("n,m", [(1, 1), (777, 9000), (100_003, 25_000), (33_333, 70_001)])
def test_block_tile_sizes(b, n, m):
    key, seed, want = _case(n, m, 21 + n, 23 + m)
    _check("block_int8", n, m, key, seed, want, block_b=b)


@pytest.mark.parametrize("n,m", [(4_000_001, 1_000_003), (3_000_000, 40_000)])
def test_block_fp8_full_chunks_all_ones(n, m):
    # All-ones key and seed: every output is the parity of n (each row meets all n key
    # bits), and every CTA of the tcgen05 kernel accumulates its whole contraction chunk
    # (16384 positions at these sizes), the largest FP32 partial sums the kernel forms.
    kw, sw = (n + 63) // 64, (n + m - 1 + 63) // 64
    key = np.full(kw, np.uint64(0xFFFFFFFFFFFFFFFF))
    seed = np.full(sw, np.uint64(0xFFFFFFFFFFFFFFFF))
    desc = pkg.pa_plan_query(n, m, binding.make_opts(path="block_fp8"))
    assert desc["path_name"] == "block_fp8"
    got, _ = run_path(n, m, key, seed, path="block_fp8")
    bits = oracle.unpack(got, m)
    assert np.all(bits == (n & 1))
    # the measured pre-rounding residual of the FP32 sums is exactly zero
    import torch
    from gpu_util import dev
    plan = pkg.Plan(n, m, path="block_fp8")
    out = torch.zeros((m + 63) // 64, dtype=torch.int64, device="cuda")
    plan.hash(dev(seed), dev(key), out)
    res, bound = plan.residual()
    plan.close()
    assert res == 0.0 and bound == 0.0
    if m % 64:
        assert int(got[-1]) >> (m % 64) == 0


@pytest.mark.parametrize("chunk", [8192, 16384, 32768])
@pytest.mark.parametrize("density", [0.97, 0.6])
def test_block_fp8_dense_full_chunks(chunk, density):
    # Where the exactness of the tensor-core sums is tight: an all-ones key and a dense seed,
    # so a CTA's count over a full chunk is about density x chunk, with random parity. At a
    # chunk of 2^15 positions the counts lie in [2^14, 2^15) (densities 0.97 and 0.6), i.e.
    # the FP32 accumulator holds count x 2^-12 in [4, 8) and needs all 15 significant bits
    # of the count; a coarser internal accumulation would drop the low bit of odd counts.
    # The whole output is compared with the oracle.
    n, m = 4 * chunk + 12_345, 2 * 32_768 + 777
    key = np.full((n + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    seed = inputs.biased_bits(n + m - 1, 4000 + chunk // 128 + int(density * 100), density)
    want = oracle.hash_full(n, m, seed, key)
    desc = pkg.pa_plan_query(n, m, binding.make_opts(path="block_fp8", tile_in=chunk))
    assert desc["path_name"] == "block_fp8" and desc["tile_in"] == chunk, desc
    import torch
    plan = pkg.Plan(n, m, path="block_fp8", tile_in=chunk)
    out = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
    plan.hash(dev(seed), dev(key), out)
    torch.cuda.synchronize()
    res, bound = plan.residual()
    st = plan.status()
    plan.close()
    got = host(out)
    bad = np.flatnonzero(got != want)
    assert st == 0 and bad.size == 0, (f"chunk {chunk} density {density}: {bad.size} words "
                                       f"differ (status {st})")
    assert res == 0.0 and bound == 0.0


def test_paper_scale_block_sampled_rows():
    # One block at the paper's upper range (Fig. 3: keys of 1e9 bits and more, l = 10%):
    # n = 1e9 + 7, m = 1e8 through the autotuned plan (the 31-bit prime: counts reach n),
    # checked on sampled rows the oracle evaluates one by one.
    n, m = 1_000_000_007, 100_000_000
    b = inputs.single_block(n, m, 31, 32)
    key, seed = b.key(), b.seed()
    got, desc = run_path(n, m, key, seed, path="auto")
    assert desc["path_name"] in ("ntt31", "ntt64")
    rng = np.random.default_rng(9)
    rows = np.unique(np.concatenate([rng.integers(0, m, 200), [0, 1, 63, 64, m - 1]]))
    want = oracle.hash_rows(n, m, seed, key, rows)
    assert np.array_equal(oracle.unpack(got, m)[rows], want), desc


def test_paper_scale_3e9_sampled_rows():
    # n = 3e9 (Fig. 3 runs to 1e10 bits), l = 10%: above both 32-bit primes, so the
    # 29-bit field takes several transform-domain sums per output tile (67 GB of spectra),
    # checked on sampled rows including output-tile edges.
    n, m = 3_000_000_019, 300_000_000
    b = inputs.single_block(n, m, 33, 34)
    key, seed = b.key(), b.seed()
    got, desc = run_path(n, m, key, seed, path="auto")
    assert desc["path_name"] == "ntt31" and desc["prime_bits"] == 29, desc
    assert desc["fd"] == 1 and desc["sum_groups"] > 1, desc
    M = desc["tile_out"]
    rng = np.random.default_rng(13)
    rows = np.unique(np.concatenate([rng.integers(0, m, 12), [0, M - 1, M, m - 1]]))
    want = oracle.hash_rows(n, m, seed, key, rows)
    assert np.array_equal(oracle.unpack(got, m)[rows], want), desc


@pytest.mark.parametrize("path,seg_in,seg_out,fd_group",
                         [("ntt31", 3, 2, 0), ("ntt31", 2, 3, 0), ("ntt31", 3, 1, 2),
                          ("ntt31", 8, 1, 0), ("ntt64", 3, 2, 0)])
def test_segmented_sums_full(path, seg_in, seg_out, fd_group):
    # Transform-domain sums run in segments over one reused spectra workspace (the paper's
    # blocks run serially, Sec. 3): 8 key tiles x 3 output tiles of 2^18 at N = 2^19,
    # forced into key segments of seg_in tiles and output slices of seg_out tiles (ragged
    # last ones), optionally with several sums per segment; compared in full.
    n, m = 2_000_007, 600_003
    key, seed, want = _case(n, m, 81, 82)
    opts = dict(log2_transform=19, tile_in=1 << 18, tile_out=1 << 18, fd_mode=2,
                seg_in=seg_in, seg_out=seg_out, fd_group=fd_group)
    desc = pkg.pa_plan_query(n, m, binding.make_opts(path=path, **opts))
    assert desc["fd"] == 1 and desc["tiles_in"] == 8 and desc["tiles_out"] == 3, desc
    assert desc["segments"] == -(-3 // seg_out) * -(-8 // seg_in), desc
    _check(path, n, m, key, seed, want, **opts)


@pytest.mark.parametrize("path,opts", [("ntt31", {}), ("ntt31", {"ntt_prime": 29}),
                                       ("ntt31", {"ntt_prime": 31}), ("ntt64", {}),
                                       ("ntt31", {"fd_group": 50}),
                                       ("ntt31", {"seg_in": 60, "seg_out": 20}),
                                       ("ntt31", {"fd_group": 40, "seg_in": 90, "seg_out": 25})])
def test_outer_convolution_sums_full(path, opts):
    # With equal key and output tiles the sums over key tiles are, bin by bin, convolutions
    # over the tile index: 123 key x 37 output tiles of 2^14 at N = 2^15 with those sums
    # forced to transforms over the tile index (one group, several groups, segments with
    # ragged slices; the 28-, 29-, 31- and 64-bit fields), compared with the oracle in full.
    n, m = 2_000_007, 600_003
    key, seed, want = _case(n, m, 91, 92)
    o = dict(log2_transform=15, tile_in=1 << 14, tile_out=1 << 14, fd_mode=2, outer_mode=2, **opts)
    desc = pkg.pa_plan_query(n, m, binding.make_opts(path=path, **o))
    assert desc["fd"] == 1 and desc["outer_log2"] > 0, desc
    _check(path, n, m, key, seed, want, **o)


@pytest.mark.parametrize("path,m,opts,logT", [("ntt31", 163_843, {}, 9), ("ntt31", 163_843, {"ntt_prime": 29}, 9),
                                              ("ntt31", 163_843, {"ntt_prime": 31}, 9),
                                              ("ntt64", 163_843, {}, 9), ("ntt31", 49_157, {"fd_group": 10}, 5)])
def test_outer_convolution_fused_stages_full(path, m, opts, logT):
    # Outer transforms of 2^9 and 2^5 points over the tile index (log2 T = 1 mod 4: the
    # first forward stage runs as the rows are loaded, the last inverse stage only on the
    # rows written out): 301 key tiles of 2^12 at N = 2^13, compared with the oracle in full.
    n = 1_228_807
    key, seed, want = _case(n, m, 93, 94)
    o = dict(log2_transform=13, tile_in=1 << 12, tile_out=1 << 12, fd_mode=2, outer_mode=2, **opts)
    desc = pkg.pa_plan_query(n, m, binding.make_opts(path=path, **o))
    assert desc["fd"] == 1 and desc["tiles_in"] == 301 and desc["outer_log2"] == logT, desc
    _check(path, n, m, key, seed, want, **o)


def test_paper_scale_1e10_segmented_sampled_rows():
    # Fig. 3's upper range: a 1e10-bit key, l = 10%, beyond the resident accumulation cap:
    # the plan runs its sums in key segments through one fixed workspace (32 GiB of spectra
    # at most), checked on sampled rows including output-tile edges.
    n, m = 10_000_000_019, 1_000_000_000
    b = inputs.single_block(n, m, 35, 36)
    key, seed = b.key(), b.seed()
    got, desc = run_path(n, m, key, seed, path="auto")
    assert desc["path_name"] == "ntt31" and desc["segments"] > 1, desc
    assert desc["workspace_bytes"] < (33 << 30), desc
    M = desc["tile_out"]
    rng = np.random.default_rng(17)
    rows = np.unique(np.concatenate([rng.integers(0, m, 20), [0, M - 1, M, m - 1]]))
    want = oracle.hash_rows(n, m, seed, key, rows)
    assert np.array_equal(oracle.unpack(got, m)[rows], want), desc


def _random_shapes(count=24, seed=2024):
    rng = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        n = int(np.exp(rng.uniform(0, np.log(300_000))))
        m = int(np.exp(rng.uniform(0, np.log(100_000))))
        if n * m <= 5e9:
            out.append((max(n, 1), max(m, 1)))
    return out


@pytest.mark.parametrize("path", PATHS + ["auto"])
@pytest.mark.parametrize("n,m", _random_shapes())
def test_random_shapes(path, n, m):
    # seeded log-uniform shapes: ragged tails of every tile, chunk and word boundary
    key, seed, want = _case(n, m, 71 + n, 73 + m)
    _check(path, n, m, key, seed, want)
