"""The lazily reduced fields' butterfly schedules (dft.cuh: lz_plan), checked on the host.

The radix-2^S groups of the 28- and 29-bit fields subtract multiples of p only where the
compile-time bound bookkeeping says a value could otherwise pass 2^32. Here the schedules
the CUDA build uses are dumped by a small host program (nvcc, the same headers) and replayed
on Python integers: every sum and difference below 2^32, every Shoup product in [0, 2p) and
congruent to the exact product, every output congruent to the plain butterflies' result and
below the bound the next round assumes (kIoDif p forward, kIoDit p inverse). Inputs sit at
and near the input bound, where an overflow would show.
"""
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1805_02372_gb300", "csrc")
M32 = 1 << 32

DUMP = r'''
#include <cstdio>
#include "dft.cuh"
using namespace pa;
template <class F, int S, bool DIF, bool Q1> void dump() {
    constexpr LzPlan<S> p = lz_plan<S>(DIF, Q1, F::kRoom, F::kIoDif, F::kIoDit);
    printf("G %d %d %d %u %d %d %d %u\n", S, DIF, Q1, F::P, F::kRoom, F::kIoDif, F::kIoDit, F::kRoot16);
    for (int s = 0; s < S; ++s)
        for (int k = 0; k < (1 << S); ++k) {
            const int half = 1 << (S - 1 - s);
            if (k & half) continue;
            printf("B %d %d %d %d %d %d %d\n", s, k, p.pa[s][k].c[0], p.pa[s][k].c[1], p.pb[s][k].c[0],
                   p.pb[s][k].c[1], p.K[s][k]);
        }
    for (int k = 0; k < (1 << S); ++k) printf("P %d %d %d\n", k, p.post[k].c[0], p.post[k].c[1]);
}
template <class F> void all() {
    dump<F, 1, true, false>(); dump<F, 2, true, false>(); dump<F, 3, true, false>();
    dump<F, 4, true, false>(); dump<F, 4, true, true>();
    dump<F, 1, false, false>(); dump<F, 2, false, false>(); dump<F, 3, false, false>();
    dump<F, 4, false, false>(); dump<F, 4, false, true>();
}
int main() { all<F29>(); all<F28>(); }
'''


@pytest.fixture(scope="module")
def schedules(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    d = tmp_path_factory.mktemp("lz")
    src, exe = d / "dump.cu", d / "dump"
    src.write_text(DUMP)
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I", CSRC, "-o", str(exe), str(src)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    groups, cur = [], None
    for line in out.splitlines():
        t = line.split()
        if t[0] == "G":
            cur = dict(S=int(t[1]), dif=t[2] == "1", q1=t[3] == "1", p=int(t[4]), room=int(t[5]),
                       iodif=int(t[6]), iodit=int(t[7]), r16=int(t[8]), B={}, P={})
            groups.append(cur)
        elif t[0] == "B":
            cur["B"][(int(t[1]), int(t[2]))] = ([int(t[3]), int(t[4])], [int(t[5]), int(t[6])], int(t[7]))
        else:
            cur["P"][int(t[1])] = [int(t[2]), int(t[3])]
    return groups


def _shoup(a, w, p):
    # the device's mul_tw: a w - floor(a floor(w 2^32 / p) / 2^32) p, mod 2^32
    q = (w << 32) // p
    r = (a * w - ((a * q) >> 32) * p) % M32
    assert r < 2 * p and (r - a * w) % p == 0
    return r


def _step(x, c, p):
    if c > 0:  # subtract c p if x >= c p
        return min(x, (x - c * p) % M32)
    if c < 0:  # Shoup's product by 1
        return _shoup(x, 1, p)
    return x


def _run(g, x, tw):
    S, p = g["S"], g["p"]
    x = list(x)
    for s in (range(S) if g["dif"] else range(S - 1, -1, -1)):
        half = 1 << (S - 1 - s)
        for k in range(1 << S):
            if k & half:
                continue
            k2 = k + half
            pa, pb, K = g["B"][(s, k)]
            for c in pa:
                x[k] = _step(x[k], c, p)
            for c in pb:
                x[k2] = _step(x[k2], c, p)
            w1 = g["q1"] and (k & (half - 1)) == 0
            if g["dif"]:
                a, b = x[k], x[k2]
                assert b <= K * p and a + b < M32 and a + K * p - b < M32
                x[k], d = a + b, a + K * p - b
                x[k2] = d if w1 else _shoup(d, tw(s, k, half), p)
            else:
                t = x[k2] if w1 else _shoup(x[k2], tw(s, k, half), p)
                a = x[k]
                assert t <= K * p and a + t < M32 and a + K * p - t < M32
                x[k], x[k2] = a + t, a + K * p - t
    for k in range(1 << S):
        for c in g["P"][k]:
            x[k] = _step(x[k], c, p)
    return x


def _plain(g, x, tw):
    S, p = g["S"], g["p"]
    x = [v % p for v in x]
    for s in (range(S) if g["dif"] else range(S - 1, -1, -1)):
        half = 1 << (S - 1 - s)
        for k in range(1 << S):
            if k & half:
                continue
            k2 = k + half
            w = 1 if (g["q1"] and (k & (half - 1)) == 0) else tw(s, k, half)
            if g["dif"]:
                x[k], x[k2] = (x[k] + x[k2]) % p, (x[k] - x[k2]) * w % p
            else:
                t = x[k2] * w % p
                x[k], x[k2] = (x[k] + t) % p, (x[k] - t) % p
    return x


def test_schedules_cover_both_fields(schedules):
    assert {g["p"] for g in schedules} == {469_762_049, 167_772_161}
    assert len(schedules) == 20
    for g in schedules:
        assert g["room"] == M32 // g["p"] and g["iodif"] == 4
    # the 28-bit field's forward radix-16 group subtracts in at most 10 places (32 for one
    # conditional subtraction per butterfly)
    g = next(g for g in schedules if g["p"] == 167_772_161 and g["S"] == 4 and g["dif"] and not g["q1"])
    steps = sum(sum(1 for c in a + b if c) for a, b, _ in g["B"].values())
    steps += sum(sum(1 for c in v if c) for v in g["P"].values())
    assert steps <= 10


def test_schedules_exact_and_bounded(schedules):
    rng = random.Random(1234)
    for g in schedules:
        p, S = g["p"], g["S"]
        io = g["iodif"] if g["dif"] else g["iodit"]
        for trial in range(400):
            tws = {}

            def tw(s, k, half):
                if g["q1"]:
                    e = (k & (half - 1)) * (8 // half)
                    return pow(g["r16"], e if g["dif"] else (16 - e) % 16, p)
                return tws.setdefault((s, k), rng.randrange(p))

            mode = trial % 3
            if mode == 0:
                x = [io * p - 1 - rng.randrange(4) for _ in range(1 << S)]
            elif mode == 1:
                x = [rng.randrange(io * p) for _ in range(1 << S)]
            else:
                x = [rng.choice([0, io * p - 1, rng.randrange(io * p)]) for _ in range(1 << S)]
            got = _run(g, x, tw)
            assert all(v < io * p for v in got), (p, S, g["dif"], g["q1"])
            assert [v % p for v in got] == _plain(g, x, tw), (p, S, g["dif"], g["q1"])
