"""The persistent NTT kernel's work lists, replayed on the host (no GPU).

`ntt_persistent` (csrc/ntt_kernel.cuh) hands out the items of its work list in list order
(one atomic ticket per CTA). An item may wait, with a bounded spin, for a dependency counter
to reach a target, and signals its own counters whether or not its wait succeeded. So a
list can never wait forever if every wait is already satisfied when the items are run one
by one in list order: whenever an item is handed out, every item before it has a CTA that
will finish it. The lists the library builds (csrc/ntt.cu, ntt_batch_build) are dumped here
by a small host program linked against the built library, for every layout it makes
(single-CTA pairs; standard four-step pairs with their spectra slots reused round-robin;
streamed, grouped, outer-convolution and segmented transform-domain sums; mixed batches
of all of them; the 28-, 29-, 31- and 64-bit fields), and replayed:

* every wait is satisfied by the items before it (no wait can run out on a correct GPU);
* every waited counter ends exactly at the target it was waited for (no producer of a
  waited-for result sits after its consumer, so no consumer can start early);
* every item's tile and sub-index are in range, and every tile's passes cover each column
  or row group exactly once;
* the spectra slot a standard pair reuses is shared only with the pair the kernel waits for
  (`slots` tiles earlier), and the transform-domain spectra lie beyond all slots;
* every spectrum an item reads or writes (standard key and window spectra, accumulated key,
  window and sum spectra, an outer convolution's slice of sums, every window a block's
  window-index table names) lies inside the workspace's spectra region;
* the decomposition (Sec. 3, Eq. Ti / Eq. Tij): every product, a standard pair or a term
  X_J W_d(I,J) of a transform-domain sum (its key spectrum, the window the block's table
  names, the sum's output rows), puts seed bit n-1+i-j under output row i and key bit j
  at the convolution index the inverse reads, with no cyclic wrap onto those rows; and the
  products of each block, over all launches of a segmented plan, tile its m x n plane of
  (row, key bit) exactly once.

Two planted mistakes, made on the host copy of the lists, must be caught: the lists run
backwards, and every seed window moved by one bit.

The wait and signal rules restated below are the kernel's: item type -> (counter, target)
waited for, and the counters it increments.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1805_02372_gb300", "csrc")

CHECKER = r'''
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <map>
#include <vector>

#include "internal.h"
#include "ntt_defs.cuh"

using namespace pa;

static int g_fail = 0;
static unsigned g_types = 0;
static bool g_reversed = false;  // replay every list backwards (the checker must object)
static bool g_shifted = false;   // move every seed window by one bit (the checker must object)
static uint64_t g_products = 0;  // products checked against the definition

// Sec. 3 decomposition: the (output rows) x (key bits) rectangle each product computes, per
// block of the list, collected over all launches of a plan
struct Rect {
    uint64_t ob, ol, kb, kl;
};
static std::map<uint32_t, std::vector<Rect>> g_rects;

// Pair (kp: key bits, wp: seed window, op: output rows and the convolution index K0 of the
// first row) of an N-point cyclic convolution: checks it against y[i] = XOR_j x[j] s[n-1+i-j].
static const char *pair_error(const TilePair &kp, const TilePair &wp, const TilePair &op,
                              uint64_t N, uint64_t n, uint64_t m) {
    if (kp.key_len == 0 || kp.key_bit0 < 0 || uint64_t(kp.key_bit0) + kp.key_len > n)
        return "key range";
    if (op.out_len == 0 || op.out_bit0 % 64 || op.out_bit0 + op.out_len > m) return "output range";
    if (kp.key_len > N || wp.win_len > N) return "input longer than the transform";
    // row i, key bit j: seed bit n-1+i-j is window position u = n-1+i-j - win_bit0, and the
    // product's coefficient k = u + (j - key_bit0) = n-1+i - key_bit0 - win_bit0
    const int64_t k0 = int64_t(n) - 1 + int64_t(op.out_bit0) - kp.key_bit0 - wp.win_bit0;
    if (k0 != int64_t(op.K0)) return "convolution index of the first row";
    const int64_t umin = k0 - int64_t(kp.key_len - 1), umax = k0 + int64_t(op.out_len) - 1;
    if (umin < 0 || umax >= int64_t(wp.win_len)) return "seed bit outside the window";
    // the linear product has key_len + win_len - 1 coefficients; cyclically, coefficient
    // k + N wraps onto k: none may land on a row that is read
    const int64_t lin = int64_t(kp.key_len) + int64_t(wp.win_len) - 1;
    if (umax + 0 >= int64_t(N) || int64_t(op.K0) + int64_t(op.out_len) > int64_t(N) ||
        lin - int64_t(N) > int64_t(op.K0))
        return "cyclic wrap onto the rows read";
    return nullptr;
}

// The rectangles of block blk tile [0, m) x [0, n) exactly once.
static const char *partition_error(const std::vector<Rect> &r, uint64_t n, uint64_t m) {
    std::map<uint64_t, uint64_t> rows, keys;
    for (const Rect &x : r) {
        if (rows.count(x.ob) && rows[x.ob] != x.ol) return "output tiles of two lengths";
        if (keys.count(x.kb) && keys[x.kb] != x.kl) return "key tiles of two lengths";
        rows[x.ob] = x.ol;
        keys[x.kb] = x.kl;
    }
    uint64_t at = 0;
    for (const auto &e : rows) {
        if (e.first != at) return "output rows not tiled";
        at += e.second;
    }
    if (at != m) return "output rows not covered";
    at = 0;
    for (const auto &e : keys) {
        if (e.first != at) return "key bits not tiled";
        at += e.second;
    }
    if (at != n) return "key bits not covered";
    std::vector<std::pair<uint64_t, uint64_t>> cells;
    for (const Rect &x : r) cells.push_back({x.ob, x.kb});
    std::sort(cells.begin(), cells.end());
    if (std::unique(cells.begin(), cells.end()) != cells.end()) return "a product computed twice";
    if (cells.size() != rows.size() * keys.size()) return "a product missing";
    return nullptr;
}

#define FAIL(...)                         \
    do {                                  \
        printf("FAIL %s: ", name);        \
        printf(__VA_ARGS__);              \
        printf("\n");                     \
        ++g_fail;                         \
        return;                           \
    } while (0)

// Counter indices: c1 [0, nt), c2 [nt, 2nt), c3 [2nt, 3nt), cfd [3nt, 3nt + nf),
// cfd1 [3nt + nf, 3nt + 2nf).
struct Lists {
    const NttTile *T;
    const FdBlock *F;
    uint64_t nt, nf, slots;
};

// The counters an item increments (false: the item's tile or block is out of range).
static bool signals(const Lists &L, uint32_t type, uint32_t ti, std::vector<uint64_t> *out) {
    const NttTile &t = L.T[ti];
    const uint64_t nt = L.nt, nf = L.nf;
    switch (type) {
        case IT_SMALL:
        case IT_FD_P3: return true;
        case IT_P1:
        case IT_FD_OUTER: out->push_back(ti); return true;
        case IT_P2:
        case IT_FD_STREAM:
        case IT_FD_INV2: out->push_back(nt + ti); return true;
        case IT_P3: out->push_back(2 * nt + ti); return true;
        case IT_FD_P1:
            if (t.fd >= nf) return false;
            out->push_back(ti);
            out->push_back(3 * nt + nf + t.fd);
            return true;
        case IT_FD_P2:
            if (t.fd >= nf) return false;
            out->push_back(3 * nt + t.fd);
            return true;
        case IT_FD_SUM: {
            if (t.fd >= nf) return false;
            const FdBlock &b = L.F[t.fd];
            if (t.out >= b.P) return false;
            const uint32_t nout = std::min<uint32_t>(kSum4Out, b.P - t.out);
            if (ti + nout > nt) return false;
            for (uint32_t i = 0; i < nout; ++i) {
                const NttTile &u = L.T[ti + i];
                if (u.fd != t.fd || u.out != t.out + i) return false;
                out->push_back(nt + ti + i);
            }
            return true;
        }
    }
    return false;
}

// The counter and target an item waits for: 1, or 0 if it does not wait, -1 if out of range.
static int waits(const Lists &L, uint32_t type, uint32_t ti, uint64_t *ctr, uint64_t *target) {
    const NttTile &t = L.T[ti];
    const uint64_t nt = L.nt, nf = L.nf;
    switch (type) {
        case IT_P1:
            if (ti < L.slots) return 0;
            *ctr = 2 * nt + ti - L.slots;
            *target = L.T[ti - L.slots].g1;
            return 1;
        case IT_P2: *ctr = ti; *target = 2ull * t.g1; return 1;
        case IT_P3:
        case IT_FD_P3: *ctr = nt + ti; *target = t.g2; return 1;
        case IT_FD_P2: *ctr = ti; *target = t.g1; return 1;
        case IT_FD_SUM:
        case IT_FD_OUTER:
            if (t.fd >= nf) return -1;
            *ctr = 3 * nt + t.fd;
            *target = L.F[t.fd].nfwd2;
            return 1;
        case IT_FD_STREAM:
            if (t.fd >= nf) return -1;
            *ctr = 3 * nt + nf + t.fd;
            *target = L.F[t.fd].nfwd1;
            return 1;
        case IT_FD_INV2:
            if (t.octr >= nt) return -1;
            *ctr = t.octr;
            *target = L.T[t.octr].g2;
            return 1;
    }
    return 0;
}

// Sub-indices of an item type on its tile: [0, range).
static uint64_t sub_range(const NttTile &t, uint32_t type) {
    switch (type) {
        case IT_SMALL: return 1;
        case IT_P1: return 2ull * t.g1;
        case IT_P3:
        case IT_FD_P1:
        case IT_FD_P3: return t.g1;
        default: return t.g2;  // P2, FD_P2, FD_SUM, FD_STREAM, FD_OUTER, FD_INV2
    }
}

static void check(const char *name, const NttBatchInfo &in, int field,
                  const std::vector<std::pair<uint64_t, uint64_t>> &shape) {
    const size_t nt = in.ntiles, nf = in.nfd, ni = in.host_items.size();
    std::vector<uint64_t> items(in.host_items);
    if (g_reversed) std::reverse(items.begin(), items.end());
    if (in.host_tiles.size() != nt * sizeof(NttTile) || in.host_fd.size() != nf * sizeof(FdBlock) ||
        ni != in.nitems || ni == 0)
        FAIL("table sizes");
    std::vector<NttTile> tiles(nt);
    if (nt) memcpy(tiles.data(), in.host_tiles.data(), nt * sizeof(NttTile));
    if (g_shifted)
        for (NttTile &t : tiles) t.p.win_bit0 += 1;
    Lists L{tiles.data(),
            reinterpret_cast<const FdBlock *>(in.host_fd.data()), nt, nf, in.slots};
    const uint64_t products0 = g_products;
    std::vector<uint64_t> fin(3 * nt + 2 * nf, 0), cnt(3 * nt + 2 * nf, 0), sig;
    // (tile, type) -> how often each sub-index occurs; FD_SUM rows counted on every sum
    // tile an item covers
    std::map<std::pair<uint32_t, uint32_t>, std::vector<uint32_t>> cover;
    auto mark = [&](uint32_t ti, uint32_t type, uint32_t sub) -> bool {
        std::vector<uint32_t> &v = cover[{ti, type}];
        const uint64_t r = sub_range(L.T[ti], type);
        if (v.empty()) v.assign(r, 0);
        if (sub >= r) return false;
        ++v[sub];
        return true;
    };
    for (size_t k = 0; k < ni; ++k) {
        const uint64_t it = items[k];
        const uint32_t type = static_cast<uint32_t>(it >> 60);
        const uint32_t ti = static_cast<uint32_t>((it >> 32) & 0x0FFFFFFFu);
        const uint32_t sub = static_cast<uint32_t>(it);
        if (type > IT_FD_INV2 || ti >= nt) FAIL("item %zu: type %u tile %u", k, type, ti);
        g_types |= 1u << type;
        sig.clear();
        if (!signals(L, type, ti, &sig)) FAIL("item %zu: signals out of range", k);
        for (uint64_t c : sig) ++fin[c];
        if (type == IT_FD_SUM) {
            for (size_t i = 0; i < sig.size(); ++i)
                if (!mark(ti + static_cast<uint32_t>(i), type, sub)) FAIL("item %zu: sum row %u", k, sub);
        } else if (!mark(ti, type, sub)) {
            FAIL("item %zu: sub %u out of range (type %u)", k, sub, type);
        }
    }
    // replay in list order
    for (size_t k = 0; k < ni; ++k) {
        const uint64_t it = items[k];
        const uint32_t type = static_cast<uint32_t>(it >> 60);
        const uint32_t ti = static_cast<uint32_t>((it >> 32) & 0x0FFFFFFFu);
        uint64_t c = 0, target = 0;
        const int w = waits(L, type, ti, &c, &target);
        if (w < 0) FAIL("item %zu: wait out of range", k);
        if (w == 1) {
            if (target == 0) FAIL("item %zu: waits for nothing (type %u)", k, type);
            if (cnt[c] < target)
                FAIL("item %zu (type %u tile %u) waits for %llu of counter %llu, %llu done before it",
                     k, type, ti, (unsigned long long)target, (unsigned long long)c,
                     (unsigned long long)cnt[c]);
            if (fin[c] != target)
                FAIL("item %zu (type %u tile %u): counter %llu ends at %llu, waited for %llu", k, type,
                     ti, (unsigned long long)c, (unsigned long long)fin[c], (unsigned long long)target);
        }
        sig.clear();
        signals(L, type, ti, &sig);
        for (uint64_t s : sig) ++cnt[s];
    }
    // each pass of each tile covers its groups exactly once; every tile is used
    std::vector<unsigned> roles(nt, 0);
    for (const auto &e : cover) {
        for (size_t s = 0; s < e.second.size(); ++s)
            if (e.second[s] != 1)
                FAIL("tile %u type %u: sub %zu covered %u times", e.first.first, e.first.second, s,
                     e.second[s]);
        roles[e.first.first] |= 1u << e.first.second;
    }
    uint64_t big_end = 0, fd_min = ~0ull;
    const unsigned fd_types = (1u << IT_FD_P1) | (1u << IT_FD_P2) | (1u << IT_FD_SUM) |
                              (1u << IT_FD_P3) | (1u << IT_FD_STREAM) | (1u << IT_FD_OUTER) |
                              (1u << IT_FD_INV2);
    for (size_t ti = 0; ti < nt; ++ti) {
        const unsigned r = roles[ti];
        const NttTile &t = L.T[ti];
        if (!r) FAIL("tile %zu is in no item", ti);
        if (r & (1u << IT_P1)) {
            if (r != ((1u << IT_P1) | (1u << IT_P2) | (1u << IT_P3))) FAIL("standard tile %zu passes %x", ti, r);
            big_end = std::max<uint64_t>(big_end, t.ws_off + (uint64_t(2) << t.logN));
        }
        if ((r & (1u << IT_FD_P1)) && t.fd < nf && L.F[t.fd].nfwd2 && !(r & (1u << IT_FD_P2)))
            FAIL("spectrum tile %zu has no forward pass 2", ti);
        if (r & (1u << IT_FD_P3)) {
            const unsigned p2 = r & ((1u << IT_FD_SUM) | (1u << IT_FD_STREAM) | (1u << IT_FD_INV2));
            if (p2 == 0 || (p2 & (p2 - 1))) FAIL("sum tile %zu pass-2 producers %x", ti, p2);
        }
        if (r & fd_types) fd_min = std::min<uint64_t>(fd_min, t.ws_off);
    }
    // spectra slots: tile ti shares its slot with ti - slots only
    const uint64_t S = L.slots;
    for (size_t b = 0; b < nt; ++b) {
        if (!(roles[b] & (1u << IT_P1))) continue;
        const NttTile &tb = L.T[b];
        const uint64_t b0 = tb.ws_off, b1 = b0 + (uint64_t(2) << tb.logN);
        if (b >= S) {
            if (!(roles[b - S] & (1u << IT_P1)) || L.T[b - S].ws_off != b0)
                FAIL("tile %zu does not reuse the slot of tile %zu", b, size_t(b - S));
        }
        for (size_t a = b >= S ? b - S + 1 : 0; a < b; ++a) {
            if (!(roles[a] & (1u << IT_P1))) continue;
            const uint64_t a0 = L.T[a].ws_off, a1 = a0 + (uint64_t(2) << L.T[a].logN);
            if (a0 < b1 && b0 < a1) FAIL("tiles %zu and %zu share spectra without a wait", a, b);
        }
    }
    if (fd_min != ~0ull && fd_min < big_end) FAIL("transform-domain spectra inside the slots");
    // every spectrum an item reads or writes lies in the workspace's spectra region
    const uint64_t elem = field == kFieldF64 ? 8 : 4, E = (in.bytes - in.off_spec) / elem;
    if (in.off_spec > in.bytes || in.counter_bytes != (3 * nt + 1 + 2 * nf) * 4)
        FAIL("workspace layout");
    std::vector<uint64_t> fdN(nf, 0);
    for (size_t ti = 0; ti < nt; ++ti) {
        const unsigned r = roles[ti];
        const NttTile &t = L.T[ti];
        const uint64_t N = uint64_t(1) << t.logN;
        uint64_t len = 0;
        if (r & (1u << IT_P1)) len = 2 * N;  // key spectrum, then the window's
        else if (r & (1u << IT_FD_OUTER)) len = uint64_t(t.nout) * N;  // the slice's sums
        else if (r & fd_types) len = N;
        if (len && t.ws_off + len > E)
            FAIL("tile %zu spectra [%llu, +%llu) beyond %llu", ti, (unsigned long long)t.ws_off,
                 (unsigned long long)len, (unsigned long long)E);
        if ((r & fd_types) && t.fd < nf) fdN[t.fd] = N;
    }
    for (size_t f = 0; f < nf; ++f) {
        const FdBlock &b = L.F[f];
        const uint64_t N = fdN[f], pairs = uint64_t(b.P) * b.Q;
        if (!N) FAIL("block %zu has no spectra", f);
        if (b.x_off + uint64_t(b.Q) * N > E) FAIL("block %zu key spectra beyond the region", f);
        if (b.wmap + pairs > in.host_wmap.size()) FAIL("block %zu window table", f);
        for (uint64_t e = b.wmap; e < b.wmap + pairs; ++e)
            if (b.w_off + (uint64_t(in.host_wmap[e]) + 1) * N > E)
                FAIL("block %zu window %u beyond the region", f, in.host_wmap[e]);
    }
    // the products: standard pairs directly; every term X_J W_d(I,J) of every sum through
    // its key spectrum, the window the block's table names and the sum's output rows
    for (size_t ti = 0; ti < nt; ++ti) {
        const NttTile &t = L.T[ti];
        if (!(roles[ti] & ((1u << IT_P1) | (1u << IT_SMALL)))) continue;
        if (t.p.blk >= shape.size()) FAIL("tile %zu block %u", ti, t.p.blk);
        const char *e = pair_error(t.p, t.p, t.p, uint64_t(1) << t.logN, shape[t.p.blk].first,
                                   shape[t.p.blk].second);
        ++g_products;
        if (e) FAIL("tile %zu: %s", ti, e);
        g_rects[t.p.blk].push_back({t.p.out_bit0, t.p.out_len, uint64_t(t.p.key_bit0), t.p.key_len});
    }
    for (size_t f = 0; f < nf; ++f) {
        const FdBlock &b = L.F[f];
        const uint64_t N = fdN[f];
        std::map<uint64_t, uint32_t> key_at, win_at;  // spectrum offset -> tile
        for (size_t ti = 0; ti < nt; ++ti) {
            const NttTile &t = L.T[ti];
            if (t.fd != f || !(roles[ti] & (1u << IT_FD_P1))) continue;
            (t.which ? win_at : key_at)[t.ws_off] = static_cast<uint32_t>(ti);
        }
        if (key_at.size() != b.Q) FAIL("block %zu: %zu key spectra for %u key tiles", f, key_at.size(), b.Q);
        for (size_t ti = 0; ti < nt; ++ti) {
            const NttTile &s = L.T[ti];
            if (s.fd != f || !(roles[ti] & (1u << IT_FD_P3))) continue;
            if (s.out >= b.P || s.jlo >= s.jhi || s.jhi > b.Q) FAIL("sum tile %zu ranges", ti);
            if (s.p.blk >= shape.size()) FAIL("sum tile %zu block %u", ti, s.p.blk);
            const uint64_t n = shape[s.p.blk].first, m = shape[s.p.blk].second;
            for (uint32_t J = s.jlo; J < s.jhi; ++J) {
                const auto k = key_at.find(b.x_off + uint64_t(J) * N);
                const uint32_t wi = in.host_wmap[b.wmap + uint64_t(s.out) * b.Q + J];
                const auto w = win_at.find(b.w_off + uint64_t(wi) * N);
                if (k == key_at.end() || w == win_at.end()) FAIL("sum tile %zu term %u: spectra", ti, J);
                const TilePair &kp = L.T[k->second].p, &wp = L.T[w->second].p;
                if (kp.blk != s.p.blk || wp.blk != s.p.blk) FAIL("sum tile %zu term %u: block", ti, J);
                const char *e = pair_error(kp, wp, s.p, N, n, m);
                ++g_products;
                if (e) FAIL("sum tile %zu (output %u) term %u: %s", ti, s.out, J, e);
                g_rects[s.p.blk].push_back({s.p.out_bit0, s.p.out_len, uint64_t(kp.key_bit0), kp.key_len});
            }
        }
    }
    printf("ok %s field %d items %zu tiles %zu fd %zu slots %llu products %llu\n", name, field,
           ni, nt, nf, (unsigned long long)S, (unsigned long long)(g_products - products0));
}

int main(int argc, char **argv) {
    g_reversed = argc > 1 && strcmp(argv[1], "reversed") == 0;
    g_shifted = argc > 1 && strcmp(argv[1], "shifted") == 0;
    char line[512], name[128] = "";
    uint32_t max_slots = 0;
    std::vector<BatchBlock> groups[kNumFields];
    // every block's products must tile its m x n plane exactly once (over all its launches)
    const auto partitioned = [&](const char *what, uint32_t blk, uint64_t n, uint64_t m) {
        const char *e = partition_error(g_rects[blk], n, m);
        if (e) {
            printf("FAIL %s: block %u: %s\n", what, blk, e);
            ++g_fail;
        }
    };
    while (fgets(line, sizeof(line), stdin)) {
        if (line[0] == 'B') {
            sscanf(line + 2, "%127s %u", name, &max_slots);
            for (auto &g : groups) g.clear();
        } else if (line[0] == 'X' || line[0] == 'Y') {  // Y: a refused plan is no failure
            unsigned long long n, m;
            pa_opts o;
            memset(&o, 0, sizeof(o));
            o.device = -1;
            int path;
            sscanf(line + 2, "%llu %llu %d %u %llu %llu %u %u %u %u %u %u", &n, &m, &path,
                   &o.log2_transform, (unsigned long long *)&o.tile_in,
                   (unsigned long long *)&o.tile_out, &o.fd_mode, &o.fd_group, &o.outer_mode,
                   &o.seg_in, &o.seg_out, &o.ntt_prime);
            o.path = path;
            PlanCfg cfg;
            const int rc = plan_resolve(n, m, &o, &cfg, false);
            if (line[0] == 'Y' && rc != PA_OK) {
                printf("refused %s rc %d\n", name, rc);
                continue;
            }
            if (rc != PA_OK || (cfg.path != PA_PATH_NTT31 && cfg.path != PA_PATH_NTT64)) {
                printf("FAIL %s: plan n=%llu m=%llu rc %d path %d\n", name, n, m, rc, cfg.path);
                ++g_fail;
                continue;
            }
            const TransformCfg &c = cfg.tr;
            if (!c.segs.empty()) {  // each segment is its own launch (seg_build's ranges)
                const uint64_t Sk = (c.tiles_in + c.seg_in - 1) / c.seg_in;
                for (uint64_t idx = 0; idx < c.segs.size(); ++idx) {
                    BatchBlock b;
                    b.index = 0;
                    b.n = n;
                    b.m = m;
                    b.tr = c;
                    b.tr.seg_in = b.tr.seg_out = 0;
                    b.tr.segs.clear();
                    b.tr.seg_base.clear();
                    const uint64_t a = idx / Sk, g = idx % Sk;
                    b.I0 = a * c.seg_out;
                    b.I1 = std::min<uint64_t>(c.tiles_out, (a + 1) * c.seg_out);
                    b.J0 = g * c.seg_in;
                    b.J1 = std::min<uint64_t>(c.tiles_in, (g + 1) * c.seg_in);
                    NttBatchInfo info;
                    char sn[200];
                    snprintf(sn, sizeof(sn), "%s/segment%llu", name, (unsigned long long)idx);
                    if (ntt_batch_build(c.field, {b}, max_slots, &info) != PA_OK) {
                        printf("FAIL %s: build\n", sn);
                        ++g_fail;
                        continue;
                    }
                    check(sn, info, c.field, {{n, m}});
                }
                partitioned(name, 0, n, m);
                g_rects.clear();
                continue;
            }
            BatchBlock b;
            b.n = n;
            b.m = m;
            b.tr = c;
            b.index = static_cast<uint32_t>(groups[c.field].size());
            groups[c.field].push_back(b);
        } else if (line[0] == 'E') {
            for (int f = 0; f < kNumFields; ++f) {
                if (groups[f].empty()) continue;
                NttBatchInfo info;
                if (ntt_batch_build(f, groups[f], max_slots, &info) != PA_OK) {
                    printf("FAIL %s: build field %d\n", name, f);
                    ++g_fail;
                    continue;
                }
                std::vector<std::pair<uint64_t, uint64_t>> shape;
                for (const BatchBlock &b : groups[f]) shape.push_back({b.n, b.m});
                g_rects.clear();
                check(name, info, f, shape);
                for (const BatchBlock &b : groups[f]) partitioned(name, b.index, b.n, b.m);
                g_rects.clear();
            }
        }
    }
    printf("types %x fails %d\n", g_types, g_fail);
    return g_fail ? 1 : 0;
}
'''

NTT31, NTT64 = 3, 2


def X(n, m, path=NTT31, k=0, L=0, M=0, fd=0, group=0, outer=0, si=0, so=0, prime=0):
    return f"X {n} {m} {path} {k} {L} {M} {fd} {group} {outer} {si} {so} {prime}"


def _batched_shapes(count, seed):
    # the batched workload's distribution: n log-uniform in [1e5, 4e6], compression 1%-50%
    import numpy as np
    rng = np.random.default_rng(seed)
    u, v = rng.random(count), rng.random(count)
    n = np.floor(1e5 * 40.0 ** u).astype(np.int64)
    m = np.maximum(1, np.floor((0.01 + 0.49 * v) * n)).astype(np.int64)
    return list(zip(n.tolist(), m.tolist()))


def _random_cases(count, seed):
    # forced geometries and options drawn at random (sizes kept to a few million bits):
    # one block per case, and every fifth case a batch of up to six blocks with the same
    # options; refused plans are fine, every plan built must pass the replay
    import random
    rng = random.Random(seed)
    out = []
    for c in range(count):
        path = rng.choice([NTT31, NTT31, NTT64])
        prime = rng.choice([0, 28, 29, 31]) if path == NTT31 else 0
        k = rng.choice([0, 0, 12, 13, 14, 15, 16, 17, 18])
        fd = rng.choice([0, 1, 2, 2])
        group = rng.choice([0, 0, 1, 2, 3, 5])
        outer = rng.choice([0, 1, 2])
        si, so = (rng.choice([0, 1, 2, 3, 5]), rng.choice([0, 1, 2, 4])) if fd == 2 and rng.random() < 0.3 else (0, 0)
        slots = rng.choice([0, 0, 4, 5, 6])
        blocks = []
        for _ in range(rng.randint(2, 6) if c % 5 == 4 else 1):
            n = int(10 ** rng.uniform(2, 6.5))
            m = max(1, int(n * rng.uniform(0.001, 0.8)))
            L = M = 0
            if k:
                N = 1 << k
                if k >= 13 and rng.random() < 0.25:
                    # equal tiles and several output tiles: the outer convolutions' shape
                    L = M = N // 2
                    n = max(n, 3 * L + rng.randint(0, L))
                    m = max(m, 2 * M + rng.randint(1, M))
                elif rng.random() < 0.5:
                    M = rng.choice([N // 2, N // 4, N // 8, 64 * rng.randint(1, max(1, N // 128))])
                    L = rng.choice([0, N - M, 32 * rng.randint(1, max(1, (N - M) // 32))])
                    if L and L + M > N:
                        L = 0
            blocks.append(f"Y {n} {m} {path} {k} {L} {M} {fd} {group} {outer} {si} {so} {prime}")
        out.append("\n".join([f"B random{c} {slots}", *blocks, "E"]))
    return "\n".join(out) + "\n"


def _cases():
    cases = []

    def case(name, slots, *blocks):
        cases.append("\n".join([f"B {name} {slots}", *blocks, "E"]))

    # one-CTA pairs (N <= 2^12) and standard four-step pairs, slots reused round-robin
    case("small", 0, X(50_003, 20_011, k=12, L=2048, M=2048, fd=1))
    for prime in (28, 29, 31):
        case(f"standard{prime}", 4, X(200_003, 60_001, k=13, L=4096, M=4096, fd=1, prime=prime))
    case("standard_slots5", 5, X(1_000_003, 150_001, k=14, L=8192, M=8192, fd=1))
    case("standard_unbounded", 0, X(300_007, 90_001, k=15, L=16384, M=16384, fd=1))
    case("standard64", 4, X(200_003, 60_001, NTT64, k=13, L=4096, M=4096, fd=1))
    # transform-domain sums: windows of every structure, grouped sums, streamed sums
    for path in (NTT31, NTT64):
        case(f"fd_equal{path}", 0, X(50_003, 20_011, path, k=13, L=4096, M=4096, fd=2))
        case(f"fd_l2m{path}", 0, X(50_003, 20_011, path, k=13, L=4096, M=2048, fd=2))
        case(f"fd_m2l{path}", 0, X(30_001, 40_003, path, k=13, L=2048, M=4096, fd=2))
        case(f"fd_ragged{path}", 0, X(40_000, 30_000, path, k=13, L=3008, M=1088, fd=2))
        case(f"streamed{path}", 0, X(50_003, 3_000, path, k=13, L=4096, M=3008, fd=2))
    case("fd_groups", 0, X(131_075, 70_001, k=14, L=8192, M=8192, fd=2, group=3))
    case("streamed_big", 0, X(1_000_003, 60_000, k=17, L=70_016, M=60_032, fd=2))
    case("fd_2to23", 0, X(20_000_003, 8_000_001, k=23, L=1 << 22, M=1 << 22, fd=2))
    # outer convolutions over the tile index, with and without groups
    case("outer", 0, X(400_003, 200_003, k=15, L=1 << 14, M=1 << 14, fd=2, outer=2))
    case("outer_groups", 0, X(400_003, 200_003, k=15, L=1 << 14, M=1 << 14, fd=2, group=5,
                               outer=2, prime=31))
    case("outer64", 0, X(100_003, 60_001, NTT64, k=13, L=4096, M=4096, fd=2, outer=2))
    # segmented sums (one launch per segment), direct and outer
    case("segmented", 0, X(2_000_007, 600_003, k=19, L=1 << 18, M=1 << 18, fd=2, si=3, so=2))
    case("segmented_outer", 0, X(1_000_003, 500_001, k=15, L=1 << 14, M=1 << 14, fd=2,
                                  outer=2, si=5, so=7))
    case("segmented64", 0, X(2_000_007, 600_003, NTT64, k=19, L=1 << 18, M=1 << 18, fd=2,
                              si=3, so=2, prime=0))
    # the planner's own choices
    case("paper_scale_1e9", 0, X(1_000_000_007, 100_000_000))
    case("table1_128M", 0, X(128 << 20, (128 << 20) // 10))
    # batches: the batched distribution (default plans, the 28-bit field), with few slots,
    # and one list mixing every layout
    case("batched64", 0, *[X(n, m) for n, m in _batched_shapes(64, 11)])
    case("batched64_slots4", 4, *[X(n, m, fd=1) for n, m in _batched_shapes(64, 12)])
    case("mixed", 4,
         X(50_003, 20_011, k=12, L=2048, M=2048, fd=1, prime=29),
         X(200_003, 60_001, k=13, L=4096, M=4096, fd=1, prime=29),
         X(50_003, 3_000, k=13, L=4096, M=3008, fd=2, prime=29),
         X(50_003, 20_011, k=13, L=4096, M=2048, fd=2, prime=29),
         X(131_075, 70_001, k=14, L=8192, M=8192, fd=2, group=3, prime=29),
         X(400_003, 200_003, k=15, L=1 << 14, M=1 << 14, fd=2, outer=2, prime=29),
         X(1_000_003, 150_001, k=14, L=8192, M=8192, fd=1, prime=29),
         X(8_191, 8_193, k=13, L=4096, M=4096, fd=2, prime=29))
    return "\n".join(cases) + "\n"


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    from paper_1805_02372_gb300 import build
    lib = build.build()
    d = tmp_path_factory.mktemp("wl")
    src, exe = d / "check.cu", d / "check"
    src.write_text(CHECKER)
    r = subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1",
                        "-gencode", "arch=compute_103a,code=compute_103a",
                        "-I", os.path.join(ROOT, "include"), "-I", CSRC, str(src), lib,
                        "-Xlinker", "-rpath=" + os.path.dirname(lib), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    return exe


def test_every_wait_is_satisfied_by_earlier_items(checker):
    r = subprocess.run([str(checker)], input=_cases(), capture_output=True, text=True,
                       timeout=600)
    out = r.stdout
    fails = [line for line in out.splitlines() if line.startswith("FAIL")]
    assert r.returncode == 0 and not fails, "\n".join(fails[:20]) + r.stderr[-2000:]
    oks = [line for line in out.splitlines() if line.startswith("ok ")]
    assert len(oks) >= 30
    # every item type of the kernel occurred (IT_SMALL .. IT_FD_INV2)
    types = int(out.splitlines()[-1].split()[1], 16)
    assert types == (1 << 11) - 1, hex(types)
    # every list's products were checked against the definition
    assert all(int(line.split()[-1]) > 0 for line in oks)
    # the segmented and batched cases produced their launches, over several fields
    assert sum(1 for line in oks if "/segment" in line) >= 6 + 6
    assert {line.split()[3] for line in oks} >= {"1", "2", "3"}


def test_replay_rejects_a_list_run_backwards(checker):
    # the same lists reversed put every consumer before its producers: every list that has
    # a wait at all must be rejected (only the one-CTA case has none)
    ok = subprocess.run([str(checker)], input=_cases(), capture_output=True, text=True,
                        timeout=600)
    bad = subprocess.run([str(checker), "reversed"], input=_cases(), capture_output=True,
                         text=True, timeout=600)
    names = [line.split()[1] for line in ok.stdout.splitlines() if line.startswith("ok ")]
    rejected = {line.split()[1].rstrip(":") for line in bad.stdout.splitlines()
                if line.startswith("FAIL") and "waits for" in line}
    assert bad.returncode == 1
    assert set(names) - rejected == {"small"}, sorted(set(names) - rejected)


def test_decomposition_rejects_a_shifted_window(checker):
    # every seed window moved by one bit: each list's products no longer read the seed bits
    # the definition names, so every case must be rejected
    ok = subprocess.run([str(checker)], input=_cases(), capture_output=True, text=True,
                        timeout=600)
    bad = subprocess.run([str(checker), "shifted"], input=_cases(), capture_output=True,
                         text=True, timeout=600)
    names = {line.split()[1] for line in ok.stdout.splitlines() if line.startswith("ok ")}
    rejected = {line.split()[1].rstrip(":") for line in bad.stdout.splitlines()
                if line.startswith("FAIL") and "convolution index" in line}
    assert bad.returncode == 1 and names and names <= rejected, sorted(names - rejected)


def test_random_geometries(checker):
    r = subprocess.run([str(checker)], input=_random_cases(400, 2024), capture_output=True,
                       text=True, timeout=900)
    lines = r.stdout.splitlines()
    fails = [line for line in lines if line.startswith("FAIL")]
    assert r.returncode == 0 and not fails, "\n".join(fails[:20]) + r.stderr[-2000:]
    oks = [line for line in lines if line.startswith("ok ")]
    refused = [line for line in lines if line.startswith("refused")]
    # most draws are plannable, and they reach every kind of item
    assert len(oks) > 300 and len(refused) < len(oks), (len(oks), len(refused))
    assert int(lines[-1].split()[1], 16) == (1 << 11) - 1
