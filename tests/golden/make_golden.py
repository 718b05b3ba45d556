"""Writes the stored expected values used by the GPU tests. Calls only the CPU oracle
(and the seeded input generator); never the CUDA library.

batched256.json: for each of the 256 blocks of the batched workload (n_i log-uniform in
[1e5, 4e6], r_i uniform in [0.01, 0.5], m_i = floor(r_i n_i)), the SHA-256 of the oracle
output words (little-endian uint64, ceil(m_i/64) words, tail bits zero).

finite_size.json: the finite-size block (n = 100,000,007 key bits from stream 1, a seed of
n + m - 1 bits from stream 2, m = 10,000,000 output bits), hashed in full by the oracle
(1e15 bit products: about two hours on eight cores). It stores the SHA-256 of all
ceil(m/64) output words and of each of 16 equal slices of them (slice k covers words
[k W / 16, (k+1) W / 16) with W = ceil(m/64)), so a mismatch names the rows it sits in.

Run: python tests/golden/make_golden.py [batched256] [finite_size]
"""
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_1805_02372_gb300 import inputs  # noqa: E402

SLICES = 16


def digest(words):
    return hashlib.sha256(words.astype("<u8").tobytes()).hexdigest()


def slice_digests(words, slices=SLICES):
    w = words.size
    return [digest(words[k * w // slices:(k + 1) * w // slices]) for k in range(slices)]


def batched256():
    out = []
    t0 = time.time()
    for i, b in enumerate(inputs.batched_blocks()):
        y = oracle.hash_full(b.n, b.m, b.seed(), b.key())
        out.append({"n": b.n, "m": b.m, "sha256": digest(y)})
        if i % 32 == 0:
            print(f"block {i}: n={b.n} m={b.m} ({time.time() - t0:.0f} s)", flush=True)
    with open(os.path.join(HERE, "batched256.json"), "w") as f:
        json.dump({"workload": "batched 256 blocks, master stream 3", "blocks": out}, f, indent=0)


def finite_size():
    b = inputs.FINITE_SIZE
    t0 = time.time()
    y = oracle.hash_full(b.n, b.m, b.seed(), b.key())
    secs = time.time() - t0
    rec = {"workload": "finite-size block, key stream 1, seed stream 2",
           "n": b.n, "m": b.m, "key_stream": b.key_stream, "seed_stream": b.seed_stream,
           "sha256": digest(y), "slices": SLICES, "slice_sha256": slice_digests(y),
           "ones": int(sum(bin(int(v)).count("1") for v in y)),
           "oracle_seconds": round(secs, 1), "oracle_threads": oracle.default_threads()}
    with open(os.path.join(HERE, "finite_size.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(f"finite_size: {secs:.0f} s, sha256 {rec['sha256']}", flush=True)


if __name__ == "__main__":
    targets = sys.argv[1:] or ["batched256"]
    for t in targets:
        {"batched256": batched256, "finite_size": finite_size}[t]()
