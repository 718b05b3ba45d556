"""The chunked shared-memory tile of the NTT's contiguous passes (dft.cuh: ColChunk), on the host.

The 32-bit fields' pass-2 and sum items keep each column of R rows in 16-byte chunks of four
rows, swizzled so that every access pattern of the rounds is free of bank conflicts. Here the
layout's own functions, compiled by nvcc from the same header, are checked for what the
kernel relies on: a one-to-one map of the C x R tile onto C R words, four consecutive rows in
one aligned 16-byte chunk, the group address generators (stride 16 and >= 256, the four
chunks of a stride-1 group) equal to the element map, column sets that start at an even
column and a multiple of 128 words addressed consistently from either base, and 32
distinct banks per wavefront for the rounds' lanes (one word per lane) and for the chunk
accesses (one 16-byte chunk per lane, eight lanes per wavefront).
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1805_02372_gb300", "csrc")

CHECK = r'''
#include <cstdio>
#include <vector>
#include "dft.cuh"
using namespace pa;

static int fails = 0;
#define CHECK(cond, ...) do { if (!(cond)) { if (fails++ < 10) { printf(__VA_ARGS__); printf("\n"); } } } while (0)

// most lanes of one wavefront on a bank: words (one per lane) or 16-byte chunks (8 lanes)
static int conflicts_words(const std::vector<int> &a) {
    int worst = 0;
    for (size_t i = 0; i < a.size(); ++i) {
        if (a[i] < 0) continue;
        int n = 0;
        for (size_t k = 0; k < a.size(); ++k)
            if (a[k] >= 0 && a[k] % 32 == a[i] % 32 && a[k] != a[i]) ++n;
        worst = n + 1 > worst ? n + 1 : worst;
    }
    return worst;
}
static int conflicts_chunks(const std::vector<int> &a) {
    int worst = 0;
    for (int ph = 0; ph < 4; ++ph)
        for (int i = 8 * ph; i < 8 * ph + 8; ++i) {
            if (a[i] < 0) continue;
            int n = 0;
            for (int k = 8 * ph; k < 8 * ph + 8; ++k)
                if (a[k] >= 0 && (a[k] / 4) % 8 == (a[i] / 4) % 8) ++n;
            worst = n > worst ? n : worst;
        }
    return worst;
}

template <int LQ, int K>
static void check_round(const ColChunk &L, int logR, int logC) {
    const int S = K == 16 ? 4 : K == 8 ? 3 : K == 4 ? 2 : 1;
    const int q = 1 << LQ, logG = logR - S, total = 1 << (logG + logC);
    for (int w0 = 0; w0 < total; w0 += 32) {
        for (int k = 0; k < K; ++k) {
            std::vector<int> lanes(32, -1);
            for (int t = 0; t < 32 && w0 + t < total; ++t) {
                const int w = w0 + t, g = w & ((1 << logG) - 1), c = w >> logG;
                const int i0 = ((g >> LQ) << (LQ + S)) + (g & (q - 1));
                int a[K];
                L.template addrs<LQ, K>(i0, c, a);
                CHECK(a[k] == L.at(i0 + k * q, c), "addrs<%d,%d> R=2^%d i0=%d c=%d k=%d", LQ, K, logR, i0, c, k);
                lanes[t] = a[k];
            }
            CHECK(conflicts_words(lanes) <= 1, "bank conflict: stride 2^%d, R=2^%d C=2^%d", LQ, logR, logC);
        }
    }
}

int main() {
    for (int logR = 6; logR <= 12; ++logR)
        for (int logC = 0; logC <= 7; ++logC) {
            const int R = 1 << logR, C = 1 << logC;
            if (R * C > 16384 || R * C < 128) continue;
            const ColChunk L = ColChunk::make(logR);
            CHECK(L.cs == R && ColChunk::words(R, C) == R * C, "sizes");
            std::vector<int> seen(R * C, 0);
            for (int c = 0; c < C; ++c)
                for (int r = 0; r < R; ++r) {
                    const int a = L.at(r, c);
                    CHECK(a >= 0 && a < R * C, "range");
                    if (a >= 0 && a < R * C) ++seen[a];
                    if ((r & 3) == 0) CHECK(a % 4 == 0, "chunk alignment");
                    else CHECK(a == L.at(r & ~3, c) + (r & 3), "chunk whole");
                }
            for (int i = 0; i < R * C; ++i) CHECK(seen[i] == 1, "bijection R=2^%d C=2^%d", logR, logC);
            for (int C0 = 2; C0 <= 8; C0 *= 2)
                if ((C0 * R) % 128 == 0)
                    for (int c = 0; c < 4; ++c)
                        for (int r = 0; r < R; r += 5) CHECK(L.at(r, C0 + c) == C0 * R + L.at(r, c), "column set");
            // the rounds dif_columns runs: logR mod 4 stages at the top, then four at a time
            const int s0 = logR & 3;
            if (s0 == 2 && logR == 6) check_round<4, 4>(L, logR, logC);
            if (s0 == 3 && logR == 7) check_round<4, 8>(L, logR, logC);
            if (logR >= 8) check_round<4, 16>(L, logR, logC);
            if (logR >= 12) check_round<8, 16>(L, logR, logC);
            if (s0 == 1 && logR == 9) check_round<8, 2>(L, logR, logC);
            if (s0 == 2 && logR == 10) check_round<8, 4>(L, logR, logC);
            if (s0 == 3 && logR == 11) check_round<8, 8>(L, logR, logC);
            // stride-1 groups: lanes on consecutive groups, four chunks each
            const int groups = (R / 16) * C;
            for (int w0 = 0; w0 < groups; w0 += 32)
                for (int u = 0; u < 4; ++u) {
                    std::vector<int> lanes(32, -1);
                    for (int t = 0; t < 32 && w0 + t < groups; ++t) {
                        const int w = w0 + t, g = w % (R / 16), c = w / (R / 16);
                        int a[4];
                        L.chunks(16 * g, c, a);
                        CHECK(a[u] == L.at(16 * g + 4 * u, c), "chunks");
                        lanes[t] = a[u];
                    }
                    CHECK(conflicts_chunks(lanes) <= 1, "chunk conflict R=2^%d C=2^%d", logR, logC);
                }
            // warp-local pairs (R >= 256): a half-warp per (column, 256-row block) pair
            if (logR >= 8) {
                const int lb = logR - 8, npairs = C << lb;
                for (int p0 = 0; p0 < npairs; p0 += 2) {
                    for (int k = 0; k < 16; ++k) {
                        std::vector<int> lanes(32, -1);
                        for (int t = 0; t < 32; ++t) {
                            const int p = p0 + (t >> 4);
                            if (p >= npairs) continue;
                            int a[16];
                            L.addrs<4, 16>(((p & ((1 << lb) - 1)) << 8) + (t & 15), p >> lb, a);
                            lanes[t] = a[k];
                        }
                        CHECK(conflicts_words(lanes) <= 1, "warp-local stride 16 conflict R=2^%d", logR);
                    }
                    for (int u = 0; u < 4; ++u) {
                        std::vector<int> lanes(32, -1);
                        for (int t = 0; t < 32; ++t) {
                            const int p = p0 + (t >> 4);
                            if (p >= npairs) continue;
                            int a[4];
                            L.chunks(((p & ((1 << lb) - 1)) << 8) + ((t & 15) << 4), p >> lb, a);
                            lanes[t] = a[u];
                        }
                        CHECK(conflicts_chunks(lanes) <= 1, "warp-local chunk conflict R=2^%d", logR);
                    }
                }
            }
            // row copies: lane on consecutive 16-byte chunks of the C R elements
            for (int t0 = 0; t0 < R * C / 4; t0 += 32) {
                std::vector<int> lanes(32, -1);
                for (int t = 0; t < 32 && t0 + t < R * C / 4; ++t) {
                    const int e = 4 * (t0 + t);
                    lanes[t] = L.at(e & (R - 1), e >> logR);
                }
                CHECK(conflicts_chunks(lanes) <= 1, "copy conflict R=2^%d C=2^%d", logR, logC);
            }
        }
    printf("fails %d\n", fails);
    return fails ? 1 : 0;
}
'''


def test_chunk_layout(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src, exe = tmp_path / "check.cu", tmp_path / "check"
    src.write_text(CHECK)
    subprocess.run([nvcc, "-std=c++17", "-O1", "--expt-relaxed-constexpr", "-I", CSRC, "-o", str(exe), str(src)],
                   check=True, capture_output=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
