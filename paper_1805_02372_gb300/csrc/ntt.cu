// Exact transform path: the tile products of the length-compatible decomposition
// (Sec. 3, Fig. 1-2, Steps 1-3) computed with number-theoretic transforms over a
// prime field instead of floating-point FFTs, so no rounding bound is needed.
//
// Decomposition. Output tile I covers rows [i0, i0+M), key tile J covers key bits
// [j0, j0+L) (L a multiple of 32, M of 64). With a[t] = x[j0+t] and the seed window
// w[u] = s[n-1+i0-j0-L+u] (positions outside the seed read as 0), output row i0+v
// receives coefficient L+v of the linear convolution a*w, and a cyclic convolution
// of size N >= L+M gives those coefficients unaliased.
//
// Combining tiles, two ways:
//   standard: each (output tile, key tile) pair is one cyclic convolution (forward
//     transforms of both inputs, pointwise product, inverse) whose bits are XORed into
//     the output (Eq. finalkey).
//   transform-domain accumulation (fd): the window depends on the pair only through
//     the offset d = i0 - j0, so each key-tile spectrum X_J and each distinct window
//     spectrum W_d is computed once; output tile I is the inverse of
//     Z_I = sum_J X_J * W_{d(I,J)}. Its coefficients are sums of at most n bit products,
//     below p, so the residue is the integer and its low bit is the XOR over key tiles.
//     With L = M the offsets take P + Q - 1 values: Q + (P + Q - 1) forward transforms
//     and P inverses replace 3 P Q transforms.
//
// Transforms. N = R1*R2 (a four-step split; R1, R2 <= 2^11) or N <= 2^12 in one CTA.
// Forward: decimation in frequency, natural input, bit-reversed spectrum; inverse:
// decimation in time from the bit-reversed spectrum, so no permutation pass exists.
// A CTA does R-point transforms on columns in shared memory, four radix-2 stages per
// shared-memory round trip (radix-16 groups in registers).
//
// Everything runs in ONE persistent launch (single blocks and batches alike): CTAs
// pull work items from a list; an item depends only on items before it in the list.
//   small  (N <= 2^12): a whole tile pair in one CTA.
//   P1     : forward pass 1 (stride R2) of a key tile or window read straight from the
//            packed bits, then the four-step twiddles.
//   P2     : forward pass 2 (contiguous rows of R2) of both spectra of a pair, the
//            pointwise product and the inverse pass 2.
//   P3     : twiddles, inverse pass 1, scale by N^-1, low bit, XOR of output bytes.
//   FD P1 / FD P2: the two forward passes of one fd spectrum (pass 2 in place).
//   FD SUM : Z_I rows = sum over key tiles of the products, then inverse pass 2.
//   FD P3  : P3 on Z_I.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <string.h>
#include <vector>

#include "ntt_defs.cuh"
#include "dft.cuh"  // shared-memory layouts (sizes of the launch)

namespace pa {

// ---------------------------------------------------------------- host tables

namespace {

uint64_t mulmod_host(uint64_t a, uint64_t b, uint64_t p) {
    return static_cast<uint64_t>((static_cast<unsigned __int128>(a) * b) % p);
}
uint64_t powmod_host(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1;
    a %= p;
    while (e) {
        if (e & 1) r = mulmod_host(r, a, p);
        a = mulmod_host(a, a, p);
        e >>= 1;
    }
    return r;
}
// Primitive 2^k-th root of unity: g^((p-1)/2^k) for a generator g of the group.
uint64_t root_of_unity(uint64_t p, const uint64_t *odd_factors, int nf, int two_adicity, int k) {
    for (uint64_t g = 2;; ++g) {
        bool ok = powmod_host(g, (p - 1) / 2, p) != 1;
        for (int i = 0; ok && i < nf; ++i) ok = powmod_host(g, (p - 1) / odd_factors[i], p) != 1;
        if (ok) return powmod_host(g, (p - 1) >> k, p);
        (void)two_adicity;
    }
}

template <class F>
struct FieldHost;
template <>
struct FieldHost<F31> {
    static uint64_t p() { return F31::P; }
    static uint64_t root(int k) {
        const uint64_t f[] = {3, 5};
        return root_of_unity(F31::P, f, 2, 27, k);
    }
    static F31::Tw tw(uint64_t w) {
        F31::Tw t;
        t.w = static_cast<uint32_t>(w);
        t.q = static_cast<uint32_t>((w << 32) / F31::P);
        return t;
    }
    // Final scale: N^-1 * 2^32 (undoes the unnormalised transforms and the Montgomery factor).
    static F31::Tw scale(int logn) {
        uint64_t ninv = powmod_host(uint64_t(1) << logn, F31::P - 2, F31::P);
        return tw(mulmod_host(ninv, (uint64_t(1) << 32) % F31::P, F31::P));
    }
};
template <>
struct FieldHost<F29> {
    static uint64_t p() { return F29::P; }
    static uint64_t root(int k) {
        const uint64_t f[] = {7};
        return root_of_unity(F29::P, f, 1, 26, k);
    }
    static F29::Tw tw(uint64_t w) {
        F29::Tw t;
        t.w = static_cast<uint32_t>(w);
        t.q = static_cast<uint32_t>((w << 32) / F29::P);
        return t;
    }
    static F29::Tw scale(int logn) {
        uint64_t ninv = powmod_host(uint64_t(1) << logn, F29::P - 2, F29::P);
        return tw(mulmod_host(ninv, (uint64_t(1) << 32) % F29::P, F29::P));
    }
};
template <>
struct FieldHost<F28> {
    static uint64_t p() { return F28::P; }
    static uint64_t root(int k) {
        const uint64_t f[] = {5};
        return root_of_unity(F28::P, f, 1, 25, k);
    }
    static F28::Tw tw(uint64_t w) {
        F28::Tw t;
        t.w = static_cast<uint32_t>(w);
        t.q = static_cast<uint32_t>((w << 32) / F28::P);
        return t;
    }
    static F28::Tw scale(int logn) {
        uint64_t ninv = powmod_host(uint64_t(1) << logn, F28::P - 2, F28::P);
        return tw(mulmod_host(ninv, (uint64_t(1) << 32) % F28::P, F28::P));
    }
};
template <>
struct FieldHost<F64> {
    static uint64_t p() { return F64::P; }
    static uint64_t root(int k) {
        const uint64_t f[] = {3, 5, 17, 257, 65537};
        return root_of_unity(F64::P, f, 5, 32, k);
    }
    static F64::Tw tw(uint64_t w) { return w; }
    static F64::Tw scale(int logn) {
        return powmod_host(uint64_t(1) << logn, F64::P - 2, F64::P);
    }
};

// Per-device tables: fwd[e] = w^e, inv[e] = w^-e for e < 2^(kLogMax-1), w of order 2^kLogMax.
std::mutex g_tab_mu;
Tables g_tabs[kNumFields][64];

template <class F>
int get_tables(int field, Tables *out) {
    int dev = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    Tables &t = g_tabs[field][dev];
    if (!t.fwd) {
        using Tw = typename F::Tw;
        const size_t half = size_t(1) << (kLogMax - 1);
        std::vector<Tw> f(half), i(half);
        const uint64_t p = FieldHost<F>::p();
        const uint64_t w = FieldHost<F>::root(kLogMax);
        const uint64_t wi = powmod_host(w, p - 2, p);
        uint64_t a = 1, b = 1;
        for (size_t e = 0; e < half; ++e) {
            f[e] = FieldHost<F>::tw(a);
            i[e] = FieldHost<F>::tw(b);
            a = mulmod_host(a, w, p);
            b = mulmod_host(b, wi, p);
        }
        // the stride-1 radix-16 groups use the field's compile-time 16th root: it must be
        // this table's (a mismatch would give wrong spectra, so refuse)
        if constexpr (HasRoot16<F>::value) {
            if (static_cast<uint64_t>(f[size_t(1) << (kLogMax - 4)].w) != F::kRoot16)
                return PA_ERR_INVALID;
        }
        // compact stage tables: block (dir, logR) holds st[h-1+j] = w_{2h}^(+-j), R-1 entries
        std::vector<Tw> st(size_t(2) * (kLogSmallMax + 1) * kStageBlock);
        for (int dir = 0; dir < 2; ++dir)
            for (int lr = 1; lr <= kLogSmallMax; ++lr)
                for (int idx = 0; idx < (1 << lr) - 1; ++idx) {
                    int lh = 0;
                    while ((2 << lh) <= idx + 1) ++lh;
                    const size_t j = size_t(idx + 1 - (1 << lh));
                    st[(size_t(dir) * (kLogSmallMax + 1) + lr) * kStageBlock + idx] =
                        (dir ? i : f)[j << (kLogMax - 1 - lh)];
                }
        void *df = nullptr, *di = nullptr, *ds = nullptr;
        cudaError_t e = cudaMalloc(&df, half * sizeof(Tw));
        if (e == cudaSuccess) e = cudaMalloc(&di, half * sizeof(Tw));
        if (e == cudaSuccess) e = cudaMalloc(&ds, st.size() * sizeof(Tw));
        if (e == cudaSuccess) e = cudaMemcpy(df, f.data(), half * sizeof(Tw), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(di, i.data(), half * sizeof(Tw), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(ds, st.data(), st.size() * sizeof(Tw), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(df);
            cudaFree(di);
            cudaFree(ds);
            return cuda_fail(e);
        }
        t.fwd = df;
        t.inv = di;
        t.stage = ds;
    }
    *out = t;
    return PA_OK;
}

}  // namespace

int ntt_tables(int field, Tables *out) {
    switch (field) {
        case kFieldF31: return get_tables<F31>(kFieldF31, out);
        case kFieldF29: return get_tables<F29>(kFieldF29, out);
        case kFieldF28: return get_tables<F28>(kFieldF28, out);
        default: return get_tables<F64>(kFieldF64, out);
    }
}

// ---------------------------------------------------------------- planning

namespace {

// Distinct window offsets I*M - J*L over I < P, J < Q (P*Q if that is no smaller).
uint64_t count_windows(uint64_t P, uint64_t Q, uint64_t M, uint64_t L) {
    if (P == 1 || Q == 1) return P * Q;
    if (L % M == 0 && L / M <= P) return P + (L / M) * (Q - 1);  // M (I - aJ): contiguous
    if (M % L == 0 && M / L <= Q) return (M / L) * (P - 1) + Q;  // L (bI - J): contiguous
    if (P * Q > kFdMaxPairs) return P * Q;
    std::vector<int64_t> d;
    d.reserve(P * Q);
    for (uint64_t I = 0; I < P; ++I)
        for (uint64_t J = 0; J < Q; ++J) d.push_back(int64_t(I * M) - int64_t(J * L));
    std::sort(d.begin(), d.end());
    return static_cast<uint64_t>(std::unique(d.begin(), d.end()) - d.begin());
}

// Distinct offsets of a P x Q segment in O(1): exact when one tile length divides the
// other (the geometries the planner builds), else the upper bound P Q. Sizes segments.
uint64_t count_windows_bound(uint64_t P, uint64_t Q, uint64_t M, uint64_t L) {
    if (P == 1 || Q == 1) return P * Q;
    if (L % M == 0) return L / M <= P ? P + (L / M) * (Q - 1) : P * Q;
    if (M % L == 0) return M / L <= Q ? (M / L) * (P - 1) + Q : P * Q;
    return P * Q;
}

// Outer convolutions for the sums of a P x Q geometry with equal tiles (window of (I, J)
// = (Q - 1) + I - J) and key tiles grouped by g: per (group, output slice) three transforms
// of T >= Ps + Qg - 1 points over the tile index for every bin, T products per bin, and
// the sums' round trip through global memory before their inverse pass 2. Returns the
// modelled cost in the units of the direct sums (3 N per (output, key tile) pair) and the
// transform size and slice, or INFINITY when a group does not fit 2^kLogOuterMax points.
double outer_cost(uint64_t P, uint64_t Q, uint64_t g, double N, uint32_t *logT, uint32_t *slice) {
    const uint64_t Qg = std::min(g, Q), maxT = uint64_t(1) << kLogOuterMax;
    if (P < 2 || Qg + 1 > maxT) return INFINITY;
    uint64_t Ps = std::min<uint64_t>(P, maxT - Qg + 1);
    const uint64_t slices = ceil_div(P, Ps);
    Ps = ceil_div(P, slices);  // balanced slices
    const uint32_t lt = std::max<uint32_t>(2, log2_ceil(Ps + Qg - 1));
    const double T = double(uint64_t(1) << lt);
    *logT = lt;
    *slice = static_cast<uint32_t>(Ps);
    // measured on the GB300 (n = 1e9, 3e9, 1e10 with l = 10%): an outer item takes about 2.3x
    // the transform units of its three T-point transforms and products, the direct sums
    // cost what their model says (n = 1e9: outer 1.8x the direct sums; 3e9: 0.74x)
    constexpr double kOuterUnits = 2.3;
    const double per = kOuterUnits * N * (T * (lt + 6) + 3.0 * T) + 2.0 * N * double(Ps);
    return double(ceil_div(Q, g) * slices) * per;
}

// The sums of an fd geometry (resident, or one segment of P x Q tiles): direct products or
// outer convolutions, whichever the model prices lower (or as forced); records the choice.
double sums_cost(uint64_t P, uint64_t Q, uint64_t g, double N, uint64_t M, uint64_t L,
                 SegChoice *seg) {
    const double direct = double(P) * double(Q) * 3.0 * N;
    if (!seg) return direct;
    seg->outer_logT = seg->outer_slice = 0;
    if (seg->outer_mode == 1 || L != M) return direct;
    uint32_t lt = 0, sl = 0;
    const double oc = outer_cost(P, Q, g, N, &lt, &sl);
    if (!(oc < INFINITY) || (seg->outer_mode != 2 && !(oc < 0.8 * direct))) return direct;
    seg->outer_logT = lt;
    seg->outer_slice = sl;
    return oc;
}

// Key tile for transform size 2^logn and output tile M: L = N - M rounded down to 32
// bits (or the forced L), at most the key rounded up to 32 bits; 0 if none fits.
uint64_t tile_in_for(uint64_t n, uint32_t logn, uint64_t M, uint64_t Lforce) {
    const uint64_t N = uint64_t(1) << logn;
    if (M == 0 || M >= N) return 0;
    uint64_t L = Lforce ? round_up(Lforce, 32) : ((N - M) / 32) * 32;
    if (L + M > N) return 0;
    const uint64_t Lneed = round_up(n, 32);
    if (!Lforce && L > Lneed) L = Lneed;
    return L;
}

}  // namespace

// Model: a standard pair costs three transforms plus a fixed per-pair overhead; under
// transform-domain accumulation each forward spectrum also makes a global round trip
// between its passes, and each (output, key tile) pair costs reading two spectra.
//
// Exactness: a coefficient read from a tile pair counts at most L bit products, one read
// from a transform-domain sum over g key tiles at most g L, so a sum covers at most
// (p - 1) / L key tiles; longer keys take several sums per output tile (one inverse
// transform each) whose output bits are XOR-merged. A streamed block has one accumulator,
// so it needs every key tile in one sum.
double ntt_geometry_cost(uint64_t n, uint64_t m, int field, uint32_t k, uint64_t M, uint64_t L,
                         uint32_t fd_mode, uint32_t fd_group, uint32_t *fd, uint64_t *windows,
                         uint32_t *kgroup, SegChoice *seg) {
    *fd = 0;
    *windows = 0;
    *kgroup = 0;
    if (seg) seg->seg_in = seg->seg_out = seg->outer_logT = seg->outer_slice = 0;
    if (k > static_cast<uint32_t>(kLogMax) || M == 0 || L == 0 || L + M > (uint64_t(1) << k))
        return INFINITY;
    const double N = double(uint64_t(1) << k);
    const uint64_t P = ceil_div(m, M), Q = ceil_div(n, L);
    const double pair = N * (k + 6) + 4096.0;
    // transforms above 2^22 run only under multi-output accumulation: their pass-2 rows
    // of 2^12 points leave no shared memory for a fused tile pair or a streamed sum
    const bool big = k > static_cast<uint32_t>(kLogMaxStd);
    const double std_units = big ? INFINITY : double(P) * double(Q);
    *windows = P * Q;
    if (k <= static_cast<uint32_t>(kLogSmallMax) || fd_mode == 1 || P * Q < 2 || P * Q > kFdMaxPairs)
        return std_units;
    const size_t elem = field == kFieldF64 ? 8 : 4;
    const uint64_t pmax = field == kFieldF64   ? ~uint64_t(0)
                          : field == kFieldF29 ? kPrimeF29 - 1
                          : field == kFieldF28 ? kPrimeF28 - 1
                                               : kPrimeF31 - 1;
    uint64_t g = std::min<uint64_t>(Q, pmax / L);
    if (fd_group) g = std::min<uint64_t>(g, fd_group);
    if (g == 0) return std_units;
    const uint64_t G = ceil_div(Q, g);  // sums per output tile
    const double tr = N * (k + 6) / 3.0;
    if (P == 1 && !big && G == 1) {
        // streamed: the forward pass 2 of each key tile and window runs inside the sum,
        // so 2Q forward transforms and one inverse replace 3Q (above 2^22, or with several
        // sums, a single output tile takes the multi-output sums below, one output per item)
        if (double(2 * Q) * N * elem > double(kFdMaxBytes)) return std_units;
        const double sc = double(Q) * (2 * tr + N + 4096.0) + tr + 4096.0;
        if (fd_mode == 2 || sc < 0.95 * std_units * pair) {
            *fd = 2;
            *windows = Q;
            return sc / pair;
        }
        return std_units;
    }
    const bool forced_seg = seg && (seg->seg_in_force || seg->seg_out_force);
    const uint64_t W = count_windows(P, Q, M, L);
    if (!forced_seg && double(Q + W + G * P) * N * elem <= double(kFdMaxBytes)) {
        const double fdc = double(Q + W) * (tr + 2 * N + 1024.0) + double(G * P) * (tr + N + 1024.0) +
                           sums_cost(P, Q, g, N, M, L, seg);
        if (fd_mode == 2 || big || fdc < 0.85 * std_units * pair) {
            *fd = 1;
            *windows = W;
            *kgroup = static_cast<uint32_t>(g);
            return fdc / pair;
        }
        if (seg) seg->outer_logT = seg->outer_slice = 0;
        return std_units;
    }
    if (!seg || fd_mode == 1) return std_units;
    // Segmented (the length-compatible scheme's blocks run serially through a fixed
    // workspace): key tiles in segments of si (one sum per output tile when si <= g),
    // output tiles in slices of so; each (slice, segment) holds its si key spectra, its
    // windows and its sums, and XORs its output bits into y (Eq. finalkey). The default
    // takes every output tile and one sum's worth of key tiles, then halves the slice and
    // the segment until the spectra fit the cap.
    const uint64_t cap = seg->seg_cap ? seg->seg_cap : kSegMaxBytes;
    uint64_t si = seg->seg_in_force ? std::min<uint64_t>(seg->seg_in_force, Q) : std::min<uint64_t>(g, Q);
    uint64_t so = seg->seg_out_force ? std::min<uint64_t>(seg->seg_out_force, P) : P;
    const auto seg_bytes = [&](uint64_t a, uint64_t b) {
        const uint64_t ws = count_windows_bound(b, a, M, L), gs = ceil_div(a, g);
        return double(a + ws + gs * b) * N * elem;
    };
    while (seg_bytes(si, so) > double(cap) && !seg->seg_out_force && so > 1) so = ceil_div(so, 2);
    while (seg_bytes(si, so) > double(cap) && !seg->seg_in_force && si > 1) si = ceil_div(si, 2);
    if (seg_bytes(si, so) > double(cap)) return std_units;
    const uint64_t So = ceil_div(P, so), Sk = ceil_div(Q, si);
    if (So * Sk > kSegMax) return std_units;
    const uint64_t ws = count_windows_bound(so, si, M, L), gs = ceil_div(si, g);
    const double segc = double(So * Sk) * (double(si + ws) * (tr + 2 * N + 1024.0) +
                                           double(gs * so) * (tr + N + 1024.0) + 4.0 * N +
                                           sums_cost(so, si, g, N, M, L, seg));
    *fd = 1;
    *windows = ws * So * Sk;
    *kgroup = static_cast<uint32_t>(g);
    seg->seg_in = static_cast<uint32_t>(si);
    seg->seg_out = static_cast<uint32_t>(so);
    return segc / pair;
}

int ntt_plan(uint64_t n, uint64_t m, int path, const pa_opts *o, TransformCfg *c) {
    *c = TransformCfg();
    // any n: the geometry keeps every count a coefficient reaches below the prime
    const uint32_t prime = o ? o->ntt_prime : 0;
    if (path == PA_PATH_NTT64) {
        if (prime) return PA_ERR_INVALID;
        c->field = kFieldF64;
    } else if (prime == 29 || prime == 0) {
        c->field = kFieldF29;
    } else if (prime == 28) {
        c->field = kFieldF28;
    } else if (prime == 31) {
        c->field = kFieldF31;
    } else {
        return PA_ERR_INVALID;
    }
    const int field = c->field;
    const uint32_t fd_mode = o ? o->fd_mode : 0;
    if (fd_mode > 2) return PA_ERR_INVALID;
    const uint32_t fd_group = o ? o->fd_group : 0;
    const uint32_t force = o ? o->log2_transform : 0;
    const uint64_t Mforce = o ? o->tile_out : 0, Lforce = o ? o->tile_in : 0;
    SegChoice seg;
    seg.seg_cap = o ? uint64_t(o->seg_cap_gib) << 30 : 0;
    seg.seg_in_force = o ? o->seg_in : 0;
    seg.seg_out_force = o ? o->seg_out : 0;
    seg.outer_mode = o ? o->outer_mode : 0;
    if (seg.outer_mode > 2) return PA_ERR_INVALID;
    double best_cost = INFINITY;
    uint32_t bk = 0, bfd = 0, bg = 0, bsi = 0, bso = 0, bot = 0, bos = 0;
    uint64_t bL = 0, bM = 0, bW = 0;
    for (uint32_t k = 5; k <= static_cast<uint32_t>(kLogMax); ++k) {
        if (force && k != force) continue;
        const uint64_t N = uint64_t(1) << k;
        uint64_t cands[24];
        int nc = 0;
        if (Mforce) {
            cands[nc++] = round_up(Mforce, 64);
        } else {
            cands[nc++] = round_up(m, 64);
            for (uint64_t f = 2; f <= 1024 && nc < 24 && N / f >= 64; f *= 2)
                cands[nc++] = round_up(N / f, 64);
        }
        for (int i = 0; i < nc; ++i) {
            uint64_t M = cands[i];
            if (M > round_up(m, 64)) M = round_up(m, 64);
            const uint64_t L = tile_in_for(n, k, M, Lforce);
            if (L == 0) continue;
            uint32_t fd = 0, g = 0;
            uint64_t W = 0;
            const double units =
                ntt_geometry_cost(n, m, field, k, M, L, fd_mode, fd_group, &fd, &W, &g, &seg);
            const double cost = units * (double(N) * (k + 6) + 4096.0);
            if (cost < best_cost) {
                best_cost = cost;
                bk = k;
                bL = L;
                bM = M;
                bfd = fd;
                bW = W;
                bg = g;
                bsi = seg.seg_in;
                bso = seg.seg_out;
                bot = seg.outer_logT;
                bos = seg.outer_slice;
            }
        }
    }
    if (!(best_cost < INFINITY)) return PA_ERR_UNSUPPORTED;
    // Default: the geometry is the 29-bit field's; a key shorter than the 28-bit prime runs
    // over that prime instead (no coefficient counts more than n bit products, so every sum
    // stays below it), whose transforms subtract less often (LazyField).
    c->field = (prime == 0 && path != PA_PATH_NTT64 && n < kPrimeF28) ? kFieldF28 : field;
    c->log2n = bk;
    c->L = bL;
    c->M = bM;
    c->tiles_in = ceil_div(n, bL);
    c->tiles_out = ceil_div(m, bM);
    c->fd = bfd;
    c->windows = bfd ? bW : 0;
    c->kgroup = bfd == 1 ? bg : 0;
    c->seg_in = bfd == 1 ? bsi : 0;
    c->seg_out = bfd == 1 ? bso : 0;
    c->outer_logT = bfd == 1 ? bot : 0;
    c->outer_slice = bfd == 1 ? bos : 0;
    if (bk <= static_cast<uint32_t>(kLogSmallMax)) {
        c->passes = 1;
        c->radix_log2[0] = bk;
    } else {
        int logR1 = 0, logR2 = 0;
        split_r(static_cast<int>(bk), &logR1, &logR2);
        c->passes = 2;
        c->radix_log2[0] = static_cast<uint32_t>(logR1);  // R1 (strided pass)
        c->radix_log2[1] = static_cast<uint32_t>(logR2);  // R2 (contiguous pass)
    }
    return PA_OK;
}

// ---------------------------------------------------------------- work lists

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

NttTile tile_shape(uint32_t logN, int field) {
    NttTile t{};
    t.logN = logN;
    if (field == kFieldF31) {
        const F31::Tw sc = FieldHost<F31>::scale(t.logN);
        memcpy(&t.scale, &sc, sizeof(sc));
    } else if (field == kFieldF29) {
        const F29::Tw sc = FieldHost<F29>::scale(t.logN);
        memcpy(&t.scale, &sc, sizeof(sc));
    } else if (field == kFieldF28) {
        const F28::Tw sc = FieldHost<F28>::scale(t.logN);
        memcpy(&t.scale, &sc, sizeof(sc));
    } else {
        const F64::Tw sc = FieldHost<F64>::scale(t.logN);
        memcpy(&t.scale, &sc, sizeof(sc));
    }
    if (logN > static_cast<uint32_t>(kLogSmallMax)) {
        const size_t elem = field == kFieldF64 ? 8 : 4;
        int logR1 = 0, logR2 = 0;
        split_r(static_cast<int>(t.logN), &logR1, &logR2);
        t.logR1 = static_cast<uint32_t>(logR1);
        t.logR2 = static_cast<uint32_t>(logR2);
        int logC1 = 0, logC2 = 0;
        pass_columns(static_cast<int>(t.logN), elem, &logC1, &logC2);
        t.logC1 = static_cast<uint32_t>(logC1);
        t.logC2 = static_cast<uint32_t>(logC2);
        t.g1 = static_cast<uint32_t>((uint64_t(1) << (t.logN - t.logR1)) >> logC1);
        t.g2 = static_cast<uint32_t>((uint64_t(1) << t.logR1) >> logC2);
    }
    return t;
}

// 1/T in the field's twiddle form (the scale of an outer convolution of T = 2^logT points).
uint64_t outer_scale(int field, uint32_t logT) {
    uint64_t bits = 0;
    if (field == kFieldF31) {
        const F31::Tw t = FieldHost<F31>::tw(powmod_host(uint64_t(1) << logT, F31::P - 2, F31::P));
        memcpy(&bits, &t, sizeof(t));
    } else if (field == kFieldF29) {
        const F29::Tw t = FieldHost<F29>::tw(powmod_host(uint64_t(1) << logT, F29::P - 2, F29::P));
        memcpy(&bits, &t, sizeof(t));
    } else if (field == kFieldF28) {
        const F28::Tw t = FieldHost<F28>::tw(powmod_host(uint64_t(1) << logT, F28::P - 2, F28::P));
        memcpy(&bits, &t, sizeof(t));
    } else {
        bits = powmod_host(uint64_t(1) << logT, F64::P - 2, F64::P);
    }
    return bits;
}

// The fd spectra and sums of one block, or of one segment of it (output tiles [I0, I1),
// key tiles [J0, J1) of the BatchBlock): Q key spectra, W window spectra, P sums (P, Q
// and every index below local to the segment), with element offsets relative to the start
// of the block's fd storage.
void build_fd(const BatchBlock &b, int field, uint32_t fd_index, std::vector<NttTile> *spectra,
              std::vector<NttTile> *sums, std::vector<NttTile> *outers, FdBlock *fb,
              std::vector<uint32_t> *wmap, uint64_t *elems) {
    const TransformCfg &c = b.tr;
    const uint64_t I0 = b.I0, I1 = b.I1 ? b.I1 : c.tiles_out;
    const uint64_t J0 = b.J0, J1 = b.J1 ? b.J1 : c.tiles_in;
    const uint64_t P = I1 - I0, Q = J1 - J0, N = uint64_t(1) << c.log2n;
    std::vector<TilePair> pairs;
    make_pairs(b.n, b.m, c, b.index, &pairs, I0, I1, J0, J1);
    // distinct offsets d = I*M - J*L, each with a representative pair
    std::vector<std::pair<int64_t, uint64_t>> d(P * Q);
    for (uint64_t I = 0; I < P; ++I)
        for (uint64_t J = 0; J < Q; ++J)
            d[I * Q + J] = {int64_t((I0 + I) * c.M) - int64_t((J0 + J) * c.L), I * Q + J};
    std::vector<std::pair<int64_t, uint64_t>> u = d;
    std::sort(u.begin(), u.end());
    u.erase(std::unique(u.begin(), u.end(),
                        [](const std::pair<int64_t, uint64_t> &a,
                           const std::pair<int64_t, uint64_t> &b2) { return a.first == b2.first; }),
            u.end());
    const uint64_t W = u.size();
    const bool streamed = c.fd == 2;
    fb->x_off = 0;
    fb->w_off = Q * N;
    fb->wmap = wmap->size();
    fb->Q = static_cast<uint32_t>(Q);
    fb->P = static_cast<uint32_t>(P);
    const NttTile shape = tile_shape(c.log2n, field);
    fb->nfwd2 = streamed ? 0u : static_cast<uint32_t>((Q + W) * shape.g2);
    fb->nfwd1 = static_cast<uint32_t>((Q + W) * shape.g1);
    const size_t w0 = wmap->size();
    for (uint64_t I = 0; I < P; ++I)
        for (uint64_t J = 0; J < Q; ++J) {
            const int64_t off = d[I * Q + J].first;
            const auto it = std::lower_bound(u.begin(), u.end(), std::make_pair(off, uint64_t(0)));
            wmap->push_back(static_cast<uint32_t>(it - u.begin()));
        }
    fb->consec = 1;
    for (uint64_t I = 0; I < P && fb->consec; ++I)
        for (uint64_t J = 0; J < Q; ++J)
            if (int64_t((*wmap)[w0 + I * Q + J]) != int64_t((*wmap)[w0]) + int64_t(I) - int64_t(J)) {
                fb->consec = 0;
                break;
            }
    for (uint64_t J = 0; J < Q; ++J) {
        NttTile t = shape;
        t.p = pairs[J];  // pair (0, J): key tile J
        t.which = 0;
        t.fd = fd_index;
        t.ws_off = J * N;
        spectra->push_back(t);
    }
    for (uint64_t w = 0; w < W; ++w) {
        NttTile t = shape;
        t.p = pairs[u[w].second];
        t.which = 1;
        t.fd = fd_index;
        t.ws_off = (Q + w) * N;
        spectra->push_back(t);
    }
    // G sums per output tile, each over at most kgroup key tiles (the counts stay below the
    // prime); sum tile g P + I covers key tiles [g kgroup, (g + 1) kgroup) of output tile I
    const uint64_t kg = (!streamed && c.kgroup) ? c.kgroup : Q;
    const uint64_t G = ceil_div(Q, kg);
    // outer convolutions need consecutive windows: window (I, J) = (Q - 1) + I - J
    fb->outer = (c.outer_logT && !streamed && fb->consec && c.L == c.M && P > 1 &&
                 (*wmap)[w0] == Q - 1) ? 1u : 0u;
    const size_t elem = field == kFieldF64 ? 8 : 4;
    const size_t sum0 = sums->size();
    for (uint64_t g = 0; g < G; ++g)
        for (uint64_t I = 0; I < P; ++I) {
            NttTile t = shape;
            t.p = pairs[I * Q];  // pair (I, 0): output tile I
            t.fd = fd_index;
            t.out = static_cast<uint32_t>(I);
            t.jlo = static_cast<uint32_t>(g * kg);
            t.jhi = static_cast<uint32_t>(std::min(Q, (g + 1) * kg));
            t.ws_off = (Q + W + g * P + I) * N;
            if (fb->outer) {
                // written by the outer items of its slice, then an inverse pass 2 item per
                // row group (the forward pass-2 shape) before the inverse pass 1
                sums->push_back(t);
                continue;
            }
            if (streamed) {
                // half the rows per sum item (key, window and accumulator columns share the
                // shared memory two columns sets use elsewhere); the sum of row group rg
                // overwrites rows rg of X_0, which only that item reads
                t.logC2 = shape.logC2 - 1;
                t.g2 = shape.g2 * 2;
                t.ws_off = 0;
            } else {
                // sum items of 2048 elements per output row group, kSum4Out outputs at a time
                t.logC2 = t.logR2 >= 11 ? 0u : 11u - t.logR2;
                t.g2 = static_cast<uint32_t>((uint64_t(1) << t.logR1) >> t.logC2);
            }
            sums->push_back(t);
        }
    if (fb->outer) {
        // one outer tile per (group, output slice); octr links them both ways (indices into
        // the `sums` and `outers` vectors; the caller makes them tile-table indices)
        const uint64_t maxT = uint64_t(1) << kLogOuterMax;
        for (uint64_t g = 0; g < G; ++g) {
            const uint64_t jlo = g * kg, jhi = std::min(Q, (g + 1) * kg), Qg = jhi - jlo;
            uint64_t Ps = std::min<uint64_t>(P, maxT - Qg + 1);
            const uint64_t slices = ceil_div(P, Ps);
            Ps = ceil_div(P, slices);
            for (uint64_t I0 = 0; I0 < P; I0 += Ps) {
                const uint64_t ns = std::min(Ps, P - I0);
                const uint32_t lt = std::max<uint32_t>(2, log2_ceil(ns + Qg - 1));
                NttTile o = shape;
                o.fd = fd_index;
                o.out = static_cast<uint32_t>(I0);
                o.nout = static_cast<uint32_t>(ns);
                o.jlo = static_cast<uint32_t>(jlo);
                o.jhi = static_cast<uint32_t>(jhi);
                o.logT = lt;
                o.logCo = static_cast<uint32_t>(outer_log_cols(static_cast<int>(lt), elem));
                o.g2 = static_cast<uint32_t>(N >> o.logCo);
                o.wb = static_cast<int32_t>((Q - 1) + I0 - jlo - (Qg - 1));
                o.ws_off = (Q + W + g * P + I0) * N;
                o.scale = outer_scale(field, lt);
                o.octr = static_cast<uint32_t>(sum0 + g * P + I0);
                for (uint64_t I = I0; I < I0 + ns; ++I)
                    (*sums)[sum0 + g * P + I].octr = static_cast<uint32_t>(outers->size());
                outers->push_back(o);
            }
        }
    }
    *elems = streamed ? (Q + W) * N : (Q + W + G * P) * N;
}

}  // namespace

int ntt_batch_build(int field, const std::vector<BatchBlock> &blocks, uint32_t max_slots,
                    NttBatchInfo *info) {
    *info = NttBatchInfo();
    if (field < 0 || field >= kNumFields) return PA_ERR_INVALID;
    info->field = field;
    const size_t elem = field == kFieldF64 ? 8 : 4, twsz = 8;
    // fd_*: blocks with accumulation over several output tiles; st_*: streamed blocks
    // (one output tile), with the range of their spectra in st_spec
    std::vector<NttTile> big, small, fd_spec, fd_sum, st_spec, st_sum, fd_outer;
    std::vector<std::pair<size_t, size_t>> st_range;
    std::vector<FdBlock> fds;
    std::vector<uint32_t> wmap;
    uint64_t fd_elems = 0;
    for (const BatchBlock &b : blocks) {
        if (b.tr.log2n > static_cast<uint32_t>(kLogMax) ||
            (b.tr.log2n > static_cast<uint32_t>(kLogMaxStd) && b.tr.fd != 1))
            return PA_ERR_INVALID;
        if (b.tr.fd) {
            const uint64_t lp = (b.I1 ? b.I1 : b.tr.tiles_out) - b.I0;
            const uint64_t lq = (b.J1 ? b.J1 : b.tr.tiles_in) - b.J0;
            if (b.tr.log2n <= static_cast<uint32_t>(kLogSmallMax) || lp * lq > kFdMaxPairs ||
                b.tr.fd > 2 ||
                (b.tr.fd == 2 && b.tr.tiles_out != 1))
                return PA_ERR_INVALID;
            const bool streamed = b.tr.fd == 2;
            std::vector<NttTile> &spec = streamed ? st_spec : fd_spec;
            std::vector<NttTile> &sum = streamed ? st_sum : fd_sum;
            const size_t s0 = spec.size(), u0 = sum.size(), o0 = fd_outer.size();
            FdBlock fb{};
            uint64_t el = 0;
            build_fd(b, field, static_cast<uint32_t>(fds.size()), &spec, &sum, &fd_outer, &fb, &wmap,
                     &el);
            for (size_t i = s0; i < spec.size(); ++i) spec[i].ws_off += fd_elems;
            for (size_t i = u0; i < sum.size(); ++i) sum[i].ws_off += fd_elems;
            for (size_t i = o0; i < fd_outer.size(); ++i) fd_outer[i].ws_off += fd_elems;
            if (streamed) st_range.push_back({s0, spec.size()});
            fb.x_off += fd_elems;
            fb.w_off += fd_elems;
            fd_elems += el;
            fds.push_back(fb);
            continue;
        }
        std::vector<TilePair> pairs;
        make_pairs(b.n, b.m, b.tr, b.index, &pairs);
        for (const TilePair &p : pairs) {
            NttTile t = tile_shape(b.tr.log2n, field);
            t.p = p;
            (t.logN <= static_cast<uint32_t>(kLogSmallMax) ? small : big).push_back(t);
        }
    }
    // largest transforms first; slots of the largest spectra size, reused round-robin
    std::stable_sort(big.begin(), big.end(),
                     [](const NttTile &a, const NttTile &b) { return a.logN > b.logN; });
    size_t slot_elems = 0;
    for (const NttTile &t : big) slot_elems = std::max(slot_elems, size_t(2) << t.logN);
    const size_t cap = size_t(4) << 30;
    size_t slots = big.size();
    if (slot_elems && slots * slot_elems * elem > cap) slots = std::max<size_t>(4, cap / (slot_elems * elem));
    // slot reuse waits on the tile `slots` earlier, whose pass 3 precedes this pass 1
    // in the work list only when slots >= 3
    if (max_slots) slots = std::min<size_t>(slots, std::max<uint32_t>(max_slots, 4));
    if (slots > big.size()) slots = big.size();
    for (size_t i = 0; i < big.size(); ++i) big[i].ws_off = (i % (slots ? slots : 1)) * slot_elems;
    const uint64_t fd_origin = uint64_t(slots) * slot_elems;  // fd storage after the slots
    for (std::vector<NttTile> *v : {&fd_spec, &fd_sum, &st_spec, &st_sum, &fd_outer})
        for (NttTile &t : *v) t.ws_off += fd_origin;
    for (FdBlock &f : fds) {
        f.x_off += fd_origin;
        f.w_off += fd_origin;
    }
    // tile table: standard big tiles (indices 0..nb-1, the slot arithmetic needs them
    // first), small tiles, fd spectra, fd sums
    std::vector<NttTile> tiles = big;
    tiles.insert(tiles.end(), small.begin(), small.end());
    const size_t i_spec = tiles.size();
    tiles.insert(tiles.end(), fd_spec.begin(), fd_spec.end());
    const size_t i_sum = tiles.size();
    tiles.insert(tiles.end(), fd_sum.begin(), fd_sum.end());
    const size_t i_sspec = tiles.size();
    tiles.insert(tiles.end(), st_spec.begin(), st_spec.end());
    const size_t i_ssum = tiles.size();
    tiles.insert(tiles.end(), st_sum.begin(), st_sum.end());
    const size_t i_outer = tiles.size();
    tiles.insert(tiles.end(), fd_outer.begin(), fd_outer.end());
    if (tiles.size() >= (size_t(1) << 28)) return PA_ERR_UNSUPPORTED;
    // outer links as tile-table indices: a sum tile of an outer block points at its outer
    // tile (whose pass-1 counter counts the outer items done), an outer tile at its first sum
    for (size_t i = 0; i < fd_sum.size(); ++i)
        if (fds[fd_sum[i].fd].outer) tiles[i_sum + i].octr = static_cast<uint32_t>(i_outer + fd_sum[i].octr);
    for (size_t i = 0; i < fd_outer.size(); ++i)
        tiles[i_outer + i].octr = static_cast<uint32_t>(i_sum + fd_outer[i].octr);
    std::vector<uint64_t> items;
    auto push = [&items](uint64_t type, uint64_t ti, uint64_t sub) {
        items.push_back((type << 60) | (ti << 32) | sub);
    };
    // fd forward passes first, so the sums near the end of the list rarely wait
    for (size_t i = 0; i < fd_spec.size(); ++i)
        for (uint32_t k = 0; k < fd_spec[i].g1; ++k) push(IT_FD_P1, i_spec + i, k);
    for (size_t i = 0; i < fd_spec.size(); ++i)
        for (uint32_t k = 0; k < fd_spec[i].g2; ++k) push(IT_FD_P2, i_spec + i, k);
    // standard tiles, software-pipelined: pass 1 of tile t, pass 2 of t-1, pass 3 of t-2
    const size_t nb = big.size();
    for (size_t t = 0; t < nb + 2; ++t) {
        if (t < nb)
            for (uint32_t k = 0; k < 2 * big[t].g1; ++k) push(IT_P1, t, k);
        if (t >= 1 && t - 1 < nb)
            for (uint32_t k = 0; k < big[t - 1].g2; ++k) push(IT_P2, t - 1, k);
        if (t >= 2 && t - 2 < nb)
            for (uint32_t k = 0; k < big[t - 2].g1; ++k) push(IT_P3, t - 2, k);
    }
    // streamed blocks, pipelined: pass 1 of all spectra of block t, the sums of block
    // t - kStreamLag, inverse pass 1 of block t - 2 kStreamLag (every streamed block has
    // its own spectra storage, so the distance costs no memory and keeps the waits short)
    constexpr size_t kStreamLag = 2;
    const size_t ns = st_sum.size();
    for (size_t t = 0; t < ns + 2 * kStreamLag; ++t) {
        if (t < ns)
            for (size_t i = st_range[t].first; i < st_range[t].second; ++i)
                for (uint32_t k = 0; k < st_spec[i].g1; ++k) push(IT_FD_P1, i_sspec + i, k);
        if (t >= kStreamLag && t - kStreamLag < ns)
            for (uint32_t k = 0; k < st_sum[t - kStreamLag].g2; ++k)
                push(IT_FD_STREAM, i_ssum + t - kStreamLag, k);
        if (t >= 2 * kStreamLag && t - 2 * kStreamLag < ns)
            for (uint32_t k = 0; k < st_sum[t - 2 * kStreamLag].g1; ++k)
                push(IT_FD_P3, i_ssum + t - 2 * kStreamLag, k);
    }
    // fd sums row group by row group (the outputs of one block share their operands'
    // rows in L2), then the inverse first passes
    {
        size_t i = 0;
        while (i < fd_sum.size()) {
            size_t j = i;
            while (j < fd_sum.size() && fd_sum[j].fd == fd_sum[i].fd) ++j;
            if (fds[fd_sum[i].fd].outer) {  // outer convolutions instead (below)
                i = j;
                continue;
            }
            // one item per row group and group of kSum4Out consecutive output tiles of one
            // group of sums (the block's sum tiles come in runs of P per group)
            const size_t P = fds[fd_sum[i].fd].P;
            for (uint32_t k = 0; k < fd_sum[i].g2; ++k)
                for (size_t g0 = i; g0 < j; g0 += P)
                    for (size_t q = g0; q < g0 + P; q += kSum4Out) push(IT_FD_SUM, i_sum + q, k);
            i = j;
        }
    }
    // outer convolutions bin block by bin block, then the inverse pass 2 of their sums
    for (size_t i = 0; i < fd_outer.size(); ++i)
        for (uint32_t k = 0; k < fd_outer[i].g2; ++k) push(IT_FD_OUTER, i_outer + i, k);
    for (size_t i = 0; i < fd_sum.size(); ++i)
        if (fds[fd_sum[i].fd].outer)
            for (uint32_t k = 0; k < fd_sum[i].g2; ++k) push(IT_FD_INV2, i_sum + i, k);
    for (size_t i = 0; i < fd_sum.size(); ++i)
        for (uint32_t k = 0; k < fd_sum[i].g1; ++k) push(IT_FD_P3, i_sum + i, k);
    for (size_t i = 0; i < small.size(); ++i) push(IT_SMALL, nb + i, 0);
    if (items.size() >= (size_t(1) << 32)) return PA_ERR_UNSUPPORTED;
    info->ntiles = tiles.size();
    info->nitems = items.size();
    info->nfd = fds.size();
    info->slots = static_cast<uint32_t>(slots ? slots : 1);
    // shared memory: the largest need among the bodies present (the contiguous passes of the
    // 32-bit fields use the unpadded chunked tile, the 64-bit field the skewed columns)
    const auto pass_words = [elem](uint32_t logR, int cols) {
        return elem == 4 ? size_t(ColChunk::words(1 << logR, cols)) : size_t(ColMajor::words(1 << logR, cols));
    };
    size_t smem = 0;
    for (const NttTile &t : small)
        smem = std::max(smem, (size_t(2) << t.logN) * twsz +
                                  size_t(ColMajor::words(1 << t.logN, 2)) * elem);
    // passes 1 and 3 (every two-pass tile): the stage table, C1 columns of R1 rows and
    // the pass-1 twiddle tables
    for (const std::vector<NttTile> *v : {&big, &fd_spec, &fd_sum, &st_spec, &st_sum})
        for (const NttTile &t : *v) {
            const int logC1 = static_cast<int>(t.logC1);
            const int seglog = logC1 - (elem == 4 ? 3 : 2);
            smem = std::max(smem, (size_t(1) << t.logR1) * twsz + (size_t(1) << (t.logR1 + logC1)) * elem +
                                      size_t(p1tw_words(static_cast<int>(t.logR1), seglog)) * elem);
        }
    // fused pass 2 of a standard pair: both stage tables, key and window rows
    for (const NttTile &t : big)
        smem = std::max(smem, 2 * (size_t(1) << t.logR2) * twsz +
                                  pass_words(t.logR2, 2 << t.logC2) * elem);
    // forward pass 2 of an fd spectrum: the forward stage table and C2 rows
    for (const NttTile &t : fd_spec)
        smem = std::max(smem, (size_t(1) << t.logR2) * twsz +
                                  pass_words(t.logR2, 1 << t.logC2) * elem);
    // fd sums: the inverse stage table and kSum4Out x C columns of R2 rows; for outer
    // blocks the inverse pass 2 of one sum (the stage table and C rows)
    for (const NttTile &t : fd_sum)
        smem = std::max(smem, (size_t(1) << t.logR2) * twsz +
                                  pass_words(t.logR2, (fds[t.fd].outer ? 1 : kSum4Out) << t.logC2) * elem);
    // outer convolutions: both stage tables of T points, the forward tile (2 C columns of
    // T rows) and the product tile (C columns)
    for (const NttTile &t : fd_outer)
        smem = std::max(smem, 2 * (size_t(1) << t.logT) * twsz +
                                  3 * (size_t(1) << (t.logT + t.logCo)) * elem);
    // streamed sums: key, window and accumulator columns, then the window indices
    for (const NttTile &t : st_sum)
        smem = std::max(smem, 2 * (size_t(1) << t.logR2) * twsz +
                                  pass_words(t.logR2, 3 << t.logC2) * elem +
                                  size_t(fds[t.fd].Q) * sizeof(uint32_t));
    info->smem = smem;
    // workspace layout
    size_t off = 0;
    info->off_tiles = off;
    off = align256(off + tiles.size() * sizeof(NttTile));
    info->off_items = off;
    off = align256(off + items.size() * sizeof(uint64_t));
    info->off_fd = off;
    off = align256(off + fds.size() * sizeof(FdBlock));
    info->off_wmap = off;
    off = align256(off + wmap.size() * sizeof(uint32_t));
    info->off_counters = off;
    info->counter_bytes = (3 * tiles.size() + 1 + 2 * fds.size()) * sizeof(uint32_t);
    off = align256(off + info->counter_bytes);
    info->off_spec = off;
    off = align256(off + (size_t(info->slots) * slot_elems + fd_elems) * elem);
    info->bytes = off;
    info->host_tiles.resize(tiles.size() * sizeof(NttTile));
    memcpy(info->host_tiles.data(), tiles.data(), info->host_tiles.size());
    info->host_fd.resize(fds.size() * sizeof(FdBlock));
    if (!fds.empty()) memcpy(info->host_fd.data(), fds.data(), info->host_fd.size());
    info->host_items = std::move(items);
    info->host_wmap = std::move(wmap);
    return PA_OK;
}

namespace {
int upload(const NttBatchInfo &info, void *ws, cudaStream_t s, bool sync) {
    char *b = static_cast<char *>(ws);
    struct Part {
        size_t off;
        const void *src;
        size_t bytes;
    } parts[] = {
        {info.off_tiles, info.host_tiles.data(), info.host_tiles.size()},
        {info.off_items, info.host_items.data(), info.host_items.size() * sizeof(uint64_t)},
        {info.off_fd, info.host_fd.data(), info.host_fd.size()},
        {info.off_wmap, info.host_wmap.data(), info.host_wmap.size() * sizeof(uint32_t)},
    };
    for (const Part &p : parts) {
        if (!p.bytes) continue;
        if (sync)
            PA_CUDA_TRY(cudaMemcpy(b + p.off, p.src, p.bytes, cudaMemcpyHostToDevice));
        else
            PA_CUDA_TRY(cudaMemcpyAsync(b + p.off, p.src, p.bytes, cudaMemcpyHostToDevice, s));
    }
    Tables t;
    return ntt_tables(info.field, &t);
}
}  // namespace

int ntt_batch_upload(const NttBatchInfo &info, void *ws, cudaStream_t s) {
    return upload(info, ws, s, false);
}

namespace {

// Work list of segment `idx` of a segmented plan: output slice idx / Sk, key segment
// idx % Sk (Sk key segments per slice).
int seg_build(uint64_t n, uint64_t m, const TransformCfg &c, uint64_t idx, NttBatchInfo *info) {
    const uint64_t Sk = ceil_div(c.tiles_in, c.seg_in);
    const uint64_t a = idx / Sk, g = idx % Sk;
    BatchBlock b;
    b.index = 0;
    b.n = n;
    b.m = m;
    b.tr = c;
    b.tr.seg_in = b.tr.seg_out = 0;
    b.tr.segs.clear();
    b.tr.seg_base.clear();
    b.I0 = a * c.seg_out;
    b.I1 = std::min<uint64_t>(c.tiles_out, (a + 1) * c.seg_out);
    b.J0 = g * c.seg_in;
    b.J1 = std::min<uint64_t>(c.tiles_in, (g + 1) * c.seg_in);
    return ntt_batch_build(c.field, std::vector<BatchBlock>{b}, 0, info);
}

// Layout of a segmented plan: each segment's tables and counters one after the other, then
// ONE spectra region, as large as the largest segment needs, that every segment reuses
// (the launches run in stream order).
int seg_layout(uint64_t n, uint64_t m, TransformCfg *c) {
    const uint64_t S = ceil_div(c->tiles_out, c->seg_out) * ceil_div(c->tiles_in, c->seg_in);
    if (S == 0 || S > kSegMax) return PA_ERR_UNSUPPORTED;
    c->segs.clear();
    c->seg_base.clear();
    size_t off = 0, spec = 0;
    for (uint64_t idx = 0; idx < S; ++idx) {
        NttBatchInfo info;
        const int rc = seg_build(n, m, *c, idx, &info);
        if (rc != PA_OK) return rc;
        c->seg_base.push_back(off);
        off = align256(off + info.off_spec);
        spec = std::max(spec, info.bytes - info.off_spec);
        c->segs.push_back(static_cast<const NttLayout &>(info));
    }
    for (uint64_t idx = 0; idx < S; ++idx) {
        c->segs[idx].off_spec = off - c->seg_base[idx];
        c->segs[idx].bytes = off + spec - c->seg_base[idx];
    }
    c->lay = c->segs[0];
    c->lay.bytes = off + spec;
    return PA_OK;
}

}  // namespace

int ntt_layout(uint64_t n, uint64_t m, int path, TransformCfg *c) {
    if (c->fd == 1 && c->seg_in && c->seg_out) return seg_layout(n, m, c);
    BatchBlock b;
    b.index = 0;
    b.n = n;
    b.m = m;
    b.tr = *c;
    NttBatchInfo info;
    const int rc = ntt_batch_build(c->field, std::vector<BatchBlock>{b}, 0, &info);
    if (rc != PA_OK) return rc;
    c->lay = static_cast<const NttLayout &>(info);
    return PA_OK;
}

int ntt_init(const PlanCfg &cfg, void *ws) {
    if (!cfg.tr.segs.empty()) {
        for (size_t idx = 0; idx < cfg.tr.segs.size(); ++idx) {
            NttBatchInfo info;
            int rc = seg_build(cfg.n, cfg.m, cfg.tr, idx, &info);
            if (rc != PA_OK) return rc;
            if (info.off_spec > cfg.tr.segs[idx].off_spec) return PA_ERR_INVALID;
            rc = upload(info, static_cast<char *>(ws) + cfg.tr.seg_base[idx], nullptr, true);
            if (rc != PA_OK) return rc;
        }
        return PA_OK;
    }
    BatchBlock b;
    b.index = 0;
    b.n = cfg.n;
    b.m = cfg.m;
    b.tr = cfg.tr;
    NttBatchInfo info;
    const int rc = ntt_batch_build(cfg.tr.field, std::vector<BatchBlock>{b}, 0, &info);
    if (rc != PA_OK) return rc;
    if (info.bytes != cfg.tr.lay.bytes) return PA_ERR_INVALID;
    return upload(info, ws, nullptr, true);
}

// ---------------------------------------------------------------- launches
namespace {
int launch_any(const NttLayout &lay, void *ws, const BlockPtrs *blks, const BlockPtrs &one,
               int *status, Prof *prof, cudaStream_t s) {
    if (lay.nitems == 0) return PA_OK;
    switch (lay.field) {
        case kFieldF31: return ntt_launch_f31(lay, ws, blks, one, status, prof, s);
        case kFieldF29: return ntt_launch_f29(lay, ws, blks, one, status, prof, s);
        case kFieldF28: return ntt_launch_f28(lay, ws, blks, one, status, prof, s);
        default: return ntt_launch_f64(lay, ws, blks, one, status, prof, s);
    }
}
}  // namespace


int ntt_batch_launch(const NttBatchInfo &info, void *ws, const void *blks, int *status, Prof *prof,
                     cudaStream_t s) {
    const BlockPtrs none{};
    return launch_any(info, ws, static_cast<const BlockPtrs *>(blks), none, status, prof, s);
}

int ntt_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
               const uint64_t *key, uint64_t *out, cudaStream_t s) {
    const BlockPtrs one{reinterpret_cast<const uint32_t *>(key), reinterpret_cast<const uint32_t *>(seed),
                        reinterpret_cast<uint32_t *>(out), cfg.n, cfg.m};
    prof_begin(prof, K_MEMSET, s);
    PA_CUDA_TRY(cudaMemsetAsync(out, 0, ceil_div(cfg.m, 64) * 8, s));
    prof_end(prof, s);
    if (!cfg.tr.segs.empty()) {
        // segments in order over the shared spectra region; each XORs its output bits
        for (size_t idx = 0; idx < cfg.tr.segs.size(); ++idx) {
            const int rc = launch_any(cfg.tr.segs[idx], static_cast<char *>(ws) + cfg.tr.seg_base[idx],
                                      nullptr, one, &hdr->status, prof, s);
            if (rc != PA_OK) return rc;
        }
        return PA_OK;
    }
    return launch_any(cfg.tr.lay, ws, nullptr, one, &hdr->status, prof, s);
}

}  // namespace pa
