"""Writes the stored expected values used by the GPU tests. Calls only the CPU oracle
(and the seeded input generator); never the CUDA library.

batched256.json: for each of the 256 blocks of the batched workload (n_i log-uniform in
[1e5, 4e6], r_i uniform in [0.01, 0.5], m_i = floor(r_i n_i)), the SHA-256 of the oracle
output words (little-endian uint64, ceil(m_i/64) words, tail bits zero).

Run: python tests/golden/make_golden.py
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


def digest(words):
    return hashlib.sha256(words.astype("<u8").tobytes()).hexdigest()


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


if __name__ == "__main__":
    batched256()
