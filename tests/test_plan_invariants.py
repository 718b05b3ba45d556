"""Exactness and coverage invariants of every plan the library accepts (host only, no GPU).

A seeded sweep of shapes and forced options through `pa_plan_query`. Whatever geometry the
planner picks or is forced to, an accepted plan must keep the conditions under which its
path is exact:

* NTT paths (Sec. 3 with an exact transform): every coefficient a product or a sum reads
  counts bit products, at most L for a tile pair and g L for a transform-domain sum over g
  key tiles, and the low bit of the residue is the hash bit only while that count is below
  the prime p. So L < p, g L <= p - 1 (several sums per output tile beyond), and a
  streamed block, with one accumulator over all key tiles, needs n < p. Key and output
  tiles fit one transform (L + M <= N), cover the key and the output, and output tiles
  start on 64-bit words. The default prime is the 28-bit one below its size, else the
  29-bit one.
* FP32 FFT (Sec. 3 with a rounded transform): the proven rounding bound of the chosen tile
  is below 1/2, so rounding recovers every count.
* FP8 tensor-core contraction: at most 2^15 products per FP32 partial sum (exact).
* Direct: one tile of the whole block.
"""
import random

import pytest

import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding

P28, P29, P31, P64 = 5 * 2 ** 25 + 1, 7 * 2 ** 26 + 1, 15 * 2 ** 27 + 1, 2 ** 64 - 2 ** 32 + 1


@pytest.fixture(scope="module")
def lib():
    from paper_1805_02372_gb300 import build
    build.build()
    return binding.load()


def _ceil(a, b):
    return -(-a // b)


def _draw(rng):
    n = int(10 ** rng.uniform(0, 7))
    m = max(1, int(n * rng.uniform(0.001, 1.0)) if rng.random() < 0.9 else rng.randint(1, 5000))
    return n, m


def _ntt_opts(rng, path):
    o = dict(path=path)
    if path == "ntt31" and rng.random() < 0.5:
        o["ntt_prime"] = rng.choice([28, 29, 31])
    if rng.random() < 0.5:
        k = rng.randint(8, 22)
        o["log2_transform"] = k
        if rng.random() < 0.5:
            N = 1 << k
            M = 64 * rng.randint(1, max(1, N // 128))
            o["tile_out"] = M
            if rng.random() < 0.5:
                o["tile_in"] = 32 * rng.randint(1, max(1, (N - M) // 32))
    o["fd_mode"] = rng.choice([0, 0, 1, 2])
    if rng.random() < 0.3:
        o["fd_group"] = rng.randint(1, 6)
    o["outer_mode"] = rng.choice([0, 1, 2])
    if o["fd_mode"] == 2 and rng.random() < 0.2:
        o["seg_in"], o["seg_out"] = rng.randint(1, 4), rng.randint(1, 4)
    return o


def _check_ntt(n, m, o, d):
    k, L, M = d["log2_transform"], d["tile_in"], d["tile_out"]
    Q, P = d["tiles_in"], d["tiles_out"]
    bits = d["prime_bits"]
    p = {28: P28, 29: P29, 31: P31, 64: P64}[bits]
    if o["path"] == "ntt64":
        assert bits == 64
    elif o.get("ntt_prime"):
        assert bits == o["ntt_prime"]
    else:
        assert bits == (28 if n < P28 else 29)
    assert L + M <= 1 << k and L > 0 and M > 0
    assert Q == _ceil(n, L) and P == _ceil(m, M)
    assert M % 64 == 0 or P == 1
    assert L < p
    if d["fd"] == 2:  # streamed: one accumulator over every key tile
        assert P == 1 and n < p
    if d["fd"] == 1:
        g = (p - 1) // L
        if o.get("fd_group"):
            g = min(g, o["fd_group"])
        if d["segments"]:
            si, so = d["seg_in"], d["seg_out"]
            assert d["segments"] == _ceil(P, so) * _ceil(Q, si)
            assert d["sum_groups"] == _ceil(Q, si) * _ceil(si, min(g, si) if g else si)
        else:
            assert d["sum_groups"] == _ceil(Q, g)
    if o.get("log2_transform"):
        assert k == o["log2_transform"]
    if o.get("tile_out"):
        assert M == min(_ceil(o["tile_out"], 64) * 64, _ceil(m, 64) * 64)


@pytest.mark.parametrize("path", ["ntt31", "ntt64"])
def test_ntt_plans_stay_exact(lib, path):
    rng = random.Random(7 if path == "ntt31" else 8)
    accepted = refused = 0
    for _ in range(250):
        n, m = _draw(rng)
        o = _ntt_opts(rng, path)
        try:
            d = pkg.pa_plan_query(n, m, binding.make_opts(**o))
        except pkg.PAError as e:
            assert e.status in (binding.PA_ERR_UNSUPPORTED, binding.PA_ERR_INVALID), (n, m, o)
            refused += 1
            continue
        accepted += 1
        assert d["n"] == n and d["m"] == m and d["path_name"] == path
        _check_ntt(n, m, o, d)
    assert accepted > 150


def test_fft_plans_stay_under_half(lib):
    rng = random.Random(9)
    accepted = 0
    for _ in range(250):
        n, m = _draw(rng)
        o = dict(path="fft")
        if rng.random() < 0.5:
            k = rng.randint(6, 14)
            o["log2_transform"] = k
            if rng.random() < 0.7:
                N = 1 << k
                o["tile_out"] = 64 * rng.randint(1, max(1, N // 128))
                o["tile_in"] = 32 * rng.randint(1, max(1, (N - o["tile_out"]) // 32))
        if rng.random() < 0.2:
            o["force_fp64"] = 1
        try:
            d = pkg.pa_plan_query(n, m, binding.make_opts(**o))
        except pkg.PAError as e:
            assert e.status in (binding.PA_ERR_PRECISION, binding.PA_ERR_UNSUPPORTED,
                                binding.PA_ERR_INVALID), (n, m, o)
            continue
        accepted += 1
        k, L, M = d["log2_transform"], d["tile_in"], d["tile_out"]
        assert L + M <= 1 << k
        assert d["tiles_in"] == _ceil(n, L) and d["tiles_out"] == _ceil(m, M)
        assert 0 <= d["rounding_bound"] < 0.5
        assert d["rounding_bound"] == pkg.pa_fft_rounding_bound(k, L, M, bool(d["fp64"]))
        if o.get("force_fp64"):
            assert d["fp64"] == 1
    assert accepted > 150


def test_block_and_direct_plans(lib):
    rng = random.Random(10)
    for _ in range(200):
        n, m = _draw(rng)
        d = pkg.pa_plan_query(n, m, binding.make_opts(path="direct"))
        assert (d["tile_in"], d["tile_out"], d["tiles_in"], d["tiles_out"]) == (n, m, 1, 1)
        d = pkg.pa_plan_query(n, m, binding.make_opts(path="block_fp8"))
        chunk, chunks = d["tile_in"], d["tiles_in"]
        assert chunk % 128 == 0 and chunk <= 1 << 15
        assert chunks * chunk >= n + 128 * 255 > (chunks - 1) * chunk
        assert d["tiles_out"] == _ceil(m, d["tile_out"])
        d = pkg.pa_plan_query(n, m, binding.make_opts(path="block_int8"))
        assert d["block_b"] in (128, 256, 512)
