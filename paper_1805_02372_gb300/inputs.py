"""Seeded synthetic inputs for the Toeplitz hash (shared by tests, bench and smoke).

This module holds no arithmetic of the hash itself: it only draws uniform bits and
the workload shapes. Both the CPU oracle and the CUDA path are fed from here.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), in its counter form: output k (k = 1, 2, ...) of the
stream started at state ``s0`` is ``mix(s0 + k * 0x9E3779B97F4A7C15 mod 2^64)``
with the published 64-bit finaliser. Being counter-based, it vectorises in numpy.

Bit packing used everywhere in this project: bit j of a string lives in 64-bit word
j >> 6 at bit position j & 63 (LSB first), words in ascending order. Bits past the
string's length inside the last word are *not* cleared here on purpose, so every
consumer is exercised on garbage tails (the hash ignores them).

The paper's inputs are corrected CV-QKD keys (Sec. 3); uniform i.i.d. bits stand in
for them, with the paper's compression ratios and lengths (Table 1, Fig. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

KEY_STREAM = 1      # "seed 1": the corrected key x
SEED_STREAM = 2     # "seed 2": the Toeplitz seed s
BATCH_MASTER = 3    # master stream of the 256-block batched workload
SERVE_MASTER = 4    # master stream of the serving workload


def splitmix64(state: int, count: int, start: int = 1) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream from ``state``."""
    k = np.arange(start, start + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(state & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(state: int, count: int, start: int = 1) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(state, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def words_for(bits: int) -> int:
    return (bits + 63) // 64


def random_bits(nbits: int, stream: int) -> np.ndarray:
    """``ceil(nbits/64)`` packed words of uniform bits (tail bits random too)."""
    return splitmix64(stream, max(words_for(nbits), 1))


def biased_bits(nbits: int, stream: int, density: float) -> np.ndarray:
    """``ceil(nbits/64)`` packed words whose bits are 1 with probability ``density``
    (bit j is 1 when output j+1 of the stream, as a double in [0, 1), is below it)."""
    nw = max(words_for(nbits), 1)
    ones = uniform01(stream, nw * 64) < density
    return np.packbits(ones.astype(np.uint8), bitorder="little").view("<u8").astype(np.uint64)


def sub_stream(master: int, index: int) -> int:
    """A per-item stream id derived from a master stream (output 1000+index)."""
    return int(splitmix64(master, 1, start=1000 + index)[0])


@dataclass(frozen=True)
class Block:
    """One hash problem: key of n bits, Toeplitz seed of n+m-1 bits, m output bits."""
    n: int
    m: int
    key_stream: int
    seed_stream: int

    def key(self) -> np.ndarray:
        return random_bits(self.n, self.key_stream)

    def seed(self) -> np.ndarray:
        return random_bits(self.n + self.m - 1, self.seed_stream)


def single_block(n: int, m: int, key_stream: int = KEY_STREAM,
                 seed_stream: int = SEED_STREAM) -> Block:
    return Block(int(n), int(m), key_stream, seed_stream)


def batched_blocks(count: int = 256, master: int = BATCH_MASTER,
                   n_lo: float = 1e5, n_hi: float = 4e6,
                   r_lo: float = 0.01, r_hi: float = 0.5) -> list[Block]:
    """The batched workload: n_i log-uniform in [n_lo, n_hi], r_i uniform in
    [r_lo, r_hi], m_i = floor(r_i * n_i) (the output length rule of Sec. 2.3),
    a fresh key and seed stream per block."""
    u = uniform01(master, count, start=1)
    v = uniform01(master, count, start=1 + count)
    blocks = []
    for i in range(count):
        n = int(math.floor(n_lo * (n_hi / n_lo) ** float(u[i])))
        r = r_lo + (r_hi - r_lo) * float(v[i])
        m = max(1, int(math.floor(r * n)))
        blocks.append(Block(n, m, sub_stream(master, 2 * i), sub_stream(master, 2 * i + 1)))
    return blocks


def serving_requests(count: int, rate_hz: float, master: int = SERVE_MASTER,
                     n_lo: float = 1e5, n_hi: float = 1e8,
                     r_lo: float = 0.01, r_hi: float = 0.5):
    """Poisson request stream: (arrival_s, Block) pairs with exponential gaps of
    mean 1/rate_hz, n log-uniform in [n_lo, n_hi], ratio uniform in [r_lo, r_hi]."""
    g = uniform01(master, count, start=1)
    u = uniform01(master, count, start=1 + count)
    v = uniform01(master, count, start=1 + 2 * count)
    t = 0.0
    out = []
    for i in range(count):
        t += -math.log(1.0 - float(g[i])) / rate_hz
        n = int(math.floor(n_lo * (n_hi / n_lo) ** float(u[i])))
        r = r_lo + (r_hi - r_lo) * float(v[i])
        m = max(1, int(math.floor(r * n)))
        out.append((t, Block(n, m, sub_stream(master, 2 * i), sub_stream(master, 2 * i + 1))))
    return out


# The named single-block workloads (sizes as stated with the method's benchmarks).
PLAIN_SINGLE = single_block(100_003, 25_000)
PLAIN_VS_TRANSFORM = [single_block(1_000_000, m) for m in (10_000, 250_000, 500_000)]
FINITE_SIZE = single_block(100_000_007, 10_000_000)
