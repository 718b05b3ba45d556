// Device side of the exact transform path: the tile bodies (bit unpacking, four-step
// passes, pointwise products, transform-domain sums, output bits) and the persistent
// kernel that runs a work list of them, plus its host launch. Included once per
// prime field by ntt_f29.cu, ntt_f31.cu and ntt_f64.cu.
#pragma once

#include <string.h>

#include "ntt_defs.cuh"
#include "dft.cuh"

namespace pa {
namespace {

// ---------------------------------------------------------------- device pieces

// Copy the compact stage table of an R-point transform (dir 0: forward, 1: inverse).
template <class F>
__device__ __forceinline__ void load_stage(typename F::Tw *st, const typename F::Tw *__restrict__ stage,
                                           int dir, int logR) {
    const typename F::Tw *src = stage + (size_t(dir) * (kLogSmallMax + 1) + logR) * kStageBlock;
    for (int idx = threadIdx.x; idx < (1 << logR) - 1; idx += blockDim.x) st[idx] = src[idx];
}

// Twiddle w^E (E < 2^kLogMax) from a half table: w^(E + 2^(kLogMax-1)) = -w^E.
template <class F>
__device__ __forceinline__ typename F::Tw tw_at(const typename F::Tw *__restrict__ tab, uint32_t E) {
    constexpr uint32_t half = 1u << (kLogMax - 1);
    if (E < half) return tab[E];
    return F::neg_tw(tab[E - half]);
}

// ---------------------------------------------------------------- tile bodies
// Each body is run by all threads of a CTA, with its stage tables already in shared
// memory; the standalone kernels and the persistent batched kernel call the same bodies.

// 32 consecutive bits of the key tile (which = 0) or window (which = 1) starting at tile
// position t; positions outside the tile or the string read as 0.
__device__ __forceinline__ uint32_t tile_bits(const TilePair &pr, const BlockPtrs &bp, int which,
                                              uint64_t t) {
    uint32_t v = 0;
    if (which == 0) {
        if (t >= pr.key_len) return 0u;
        const uint64_t pos = uint64_t(pr.key_bit0) + t;
        const uint64_t kw = 2 * ((bp.n + 63) >> 6);
        v = bits32_at(bp.key32, kw, static_cast<int64_t>(pos));
        const uint64_t left = pr.key_len - t;  // valid bits from t
        if (left < 32) v &= (1u << left) - 1u;
    } else {
        if (t >= pr.win_len) return 0u;
        const int64_t pos = pr.win_bit0 + static_cast<int64_t>(t);
        const uint64_t sl = bp.n + bp.m - 1;  // seed length
        const uint64_t sw = 2 * ((sl + 63) >> 6);
        v = bits32_at(bp.seed32, sw, pos);
        // positions >= seed length or >= window length read as 0 (< 0 handled by bits32_at)
        const int64_t lim1 = static_cast<int64_t>(sl) - pos;
        const int64_t lim2 = static_cast<int64_t>(pr.win_len - t);
        const int64_t lim = lim1 < lim2 ? lim1 : lim2;
        if (lim <= 0) return 0u;
        if (lim < 32) v &= (1u << lim) - 1u;
    }
    return v;
}

// Whole transform of size 2^logN <= 2^12 in shared memory for one tile.
template <class F>
__device__ __forceinline__ void body_small(typename F::T *sm, const typename F::Tw *stf, const typename F::Tw *sti,
                           const TilePair &pr, const BlockPtrs &bp, int logN, typename F::Tw scale) {
    using T = typename F::T;
    const int N = 1 << logN;
    const ColMajor lay{ColMajor::stride(N)};
    // 32 tile positions per thread from one or two 32-bit words of each input
    for (int t0 = threadIdx.x * 32; t0 < N; t0 += blockDim.x * 32) {
        const uint32_t kb = tile_bits(pr, bp, 0, t0), wb = tile_bits(pr, bp, 1, t0);
#pragma unroll 8
        for (int k = 0; k < 32; ++k) {
            sm[lay.at(t0 + k, 0)] = (kb >> k) & 1u;
            sm[lay.at(t0 + k, 1)] = (wb >> k) & 1u;
        }
    }
    __syncthreads();
    const auto mul = [](T a, T b) { return F::mont(a, b); };
    if (logN >= 4) {
        dif_columns_head<F, false>(sm, lay, logN, 1, stf);
        product_round<F>(sm, lay, logN, 0, stf, sti, mul);
        dit_columns_tail<F, false>(sm + lay.cs, lay, logN, 0, sti);
    } else {
        dif_columns<F, false>(sm, lay, logN, 1, stf);
        for (int t = threadIdx.x; t < N; t += blockDim.x)
            sm[lay.at(t, 1)] = F::mont(sm[lay.at(t, 0)], sm[lay.at(t, 1)]);
        __syncthreads();
        dit_columns<F, false>(sm + lay.cs, lay, logN, 0, sti);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nw = (pr.out_len + 31) / 32;
    for (uint32_t w = warp; w < nw; w += blockDim.x / 32) {
        const uint32_t v = w * 32 + lane;
        uint32_t bit = 0;
        if (v < pr.out_len) bit = F::low_bit(F::mul_tw(sm[lay.at(pr.K0 + v, 1)], scale));
        const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
        if (lane == 0 && word) atomicXor(bp.out32 + (pr.out_bit0 >> 5) + w, word);
    }
    __syncthreads();
}

// A 32-byte row segment of a RowMajor tile moves as two 16-byte halves, the half
// (lane >> 2) & 1 first: the eight lanes of a quarter warp then touch eight distinct
// 16-byte bank groups for every row width (C = 8: two aligned row quads; C = 16, 32:
// rows differing in the slot bit the half separates; C >= 64: segments sg and sg + 4).
template <class T>
__device__ __forceinline__ void seg_store(T *p, const T (&x)[32 / sizeof(T)]) {
    constexpr int H = 16 / sizeof(T);
    const uint32_t h = (threadIdx.x >> 2) & 1u;
    const uint4 a = *reinterpret_cast<const uint4 *>(&x[0]);
    const uint4 b = *reinterpret_cast<const uint4 *>(&x[H]);
    uint4 *d = reinterpret_cast<uint4 *>(p);
    d[h] = h ? b : a;
    d[h ^ 1u] = h ? a : b;
}
template <class T>
__device__ __forceinline__ void seg_load(T (&x)[32 / sizeof(T)], const T *p) {
    constexpr int H = 16 / sizeof(T);
    const uint32_t h = (threadIdx.x >> 2) & 1u;
    const uint4 *s = reinterpret_cast<const uint4 *>(p);
    const uint4 f = s[h], g = s[h ^ 1u];
    *reinterpret_cast<uint4 *>(&x[0]) = h ? g : f;
    *reinterpret_cast<uint4 *>(&x[H]) = h ? f : g;
}

// 32 bytes to global memory with one 256-bit store, cached in L2 only (p 32-byte aligned):
// a lane writes a whole sector.
__device__ __forceinline__ void stcg256(void *p, const void *v) {
    const uint32_t *w = static_cast<const uint32_t *>(v);
    asm volatile("st.global.cg.v8.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(p), "r"(w[0]),
                 "r"(w[1]), "r"(w[2]), "r"(w[3]), "r"(w[4]), "r"(w[5]), "r"(w[6]), "r"(w[7])
                 : "memory");
}

// Global loads a thread keeps in flight before storing them to shared memory.
constexpr int kLoadBatch = 4;
// Row segments whose pass-1 twiddles a thread forms at once.
constexpr int kTwBatch = 2;

// Asynchronous global -> shared copies (no registers held while they are in flight);
// cp_async_wait_all waits for this thread's copies, a barrier then publishes them.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Tile layout of the contiguous passes (pass 2 and the transform-domain sums): 32-bit
// fields keep 16-byte chunks whole (ColChunk: rows staged and stored 16 bytes at a time),
// the 64-bit field keeps the skewed columns.
template <class T>
struct PassLay {
    using type = ColMajor;
    static __device__ __forceinline__ ColMajor make(int logR) { return ColMajor{ColMajor::stride(1 << logR)}; }
};
template <>
struct PassLay<uint32_t> {
    using type = ColChunk;
    static __device__ __forceinline__ ColChunk make(int logR) { return ColChunk::make(logR); }
};

// Rows of a 32-bit tile from global memory (element e of g is row e & (R - 1) of shared
// column c0 + (e >> logR)) by 16-byte asynchronous copies, one chunk per lane; the caller
// waits (cp_async_wait_all) and synchronises.
template <class T>
__device__ __forceinline__ void stage_rows(T *sm, const ColChunk &lay, int c0, const T *__restrict__ g, int cnt,
                                           int logR) {
    static_assert(sizeof(T) == 4, "chunked tiles hold 32-bit elements");
    const int R = 1 << logR;
    for (int e = threadIdx.x * 4; e < cnt; e += blockDim.x * 4)
        cp_async16(sm + lay.at(e & (R - 1), c0 + (e >> logR)), g + e);
}
// The reverse: columns c0 .. of the shared tile to global rows, 16 bytes per lane.
template <class T, class Lay>
__device__ __forceinline__ void store_rows(T *__restrict__ g, const T *sm, const Lay &lay, int c0, int cnt,
                                           int logR) {
    const int R = 1 << logR;
    constexpr int V = 16 / sizeof(T);
    for (int e = threadIdx.x * V; e < cnt; e += blockDim.x * V) {
        const int c = c0 + (e >> logR), r = e & (R - 1);
        uint4 ov;
        if constexpr (sizeof(T) == 4) {
            ov = *reinterpret_cast<const uint4 *>(sm + lay.at(r, c));
        } else {
            T *os = reinterpret_cast<T *>(&ov);
#pragma unroll
            for (int k = 0; k < V; ++k) os[k] = sm[lay.at(r + k, c)];
        }
        __stcg(reinterpret_cast<uint4 *>(g + e), ov);
    }
}

// Pass-1 twiddles (forward and inverse items) without a table lookup per row. Row r holds
// frequency f = brev(r) = 32 fh + fl, and segment sg starts at column t0 = c0 + sg SEG, so
// w^(t0 f) = w^(t0 fl) w^(32 t0 fh) and w^f = w^fl w^(32 fh): per segment column the
// tables A[fl] = w^(t0 fl), B[fh] = w^(32 t0 fh), and once C[fl] = w^fl, D[fh] = w^(32 fh),
// all in full form, give every row's first twiddle and step with one product each.
// Layout (F::T): per sg, A (32) then B (R1 / 32); then C, D.
template <class F>
__device__ void p1tw_build(typename F::T *tb, const typename F::Tw *__restrict__ tab, uint64_t c0,
                           int seg, int seglog, int logR1, int logN) {
    const int per = 32 + (1 << (logR1 - 5));
    const int total = p1tw_words(logR1, seglog);
    const int sh = kLogMax - logN;
    const uint64_t mask = (uint64_t(1) << logN) - 1;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int sg = i / per, k = i - sg * per;
        const uint64_t t0 = sg < (1 << seglog) ? c0 + uint64_t(sg) * seg : 1;
        const uint64_t e = (k < 32 ? t0 * uint64_t(k) : t0 * 32 * uint64_t(k - 32)) & mask;
        tb[i] = F::full_form(tw_at<F>(tab, static_cast<uint32_t>(e << sh)));
    }
}

// x[c] *= base step^c for c < SEG (twiddles in full form): the twiddles are formed as a
// tree (w[c + b] = w[c] step^b, step^b by squaring), log2 SEG products deep instead of
// SEG - 1, so the rows of a thread overlap their latencies.
template <class F, int SEG>
__device__ __forceinline__ void twiddle_segment(typename F::T (&x)[SEG], typename F::T base,
                                                typename F::T step) {
    using T = typename F::T;
    T w[SEG];
    w[0] = base;
    T sp = step;
#pragma unroll
    for (int b = 1; b < SEG; b <<= 1) {
#pragma unroll
        for (int c = 0; c < b; ++c) w[c + b] = F::mul_full(w[c], sp);
        if (2 * b < SEG) sp = F::mul_full(sp, sp);
    }
#pragma unroll
    for (int c = 0; c < SEG; ++c) x[c] = F::mul_full(x[c], w[c]);
}

// Pass 1 forward on column group cg (C = 2^logC columns at stride S1 = N / R1); each
// thread handles 32-byte row segments (SEG columns).
template <class F>
__device__ __forceinline__ void body_fwd_first(typename F::T *sm, const typename F::Tw *st, const TilePair &pr,
                               const BlockPtrs &bp, int which, uint64_t cg, int logN, int logR1,
                               int logC, typename F::T *__restrict__ dst,
                               const typename F::Tw *__restrict__ tfwd) {
    using T = typename F::T;
    constexpr int SEG = 32 / sizeof(T), logSEG = sizeof(T) == 4 ? 3 : 2;
    const int R1 = 1 << logR1, logS = logN - logR1, C = 1 << logC;
    const uint64_t c0 = cg << logC;
    const RowMajor lay{logC};
    const int seglog = logC - logSEG;  // segments per row (log2)
    T *tb = sm + (R1 << logC);         // pass-1 twiddle tables (p1tw_build)
    // up to kLoadBatch segments per thread: every load issued before the first store, and
    // the twiddle tables (root-table lookups) built while the first batch is in flight
    bool built = false;
    for (int e0 = threadIdx.x; e0 < (R1 << seglog); e0 += kLoadBatch * blockDim.x) {
        uint32_t bits[kLoadBatch];
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
            bits[u] = e < (R1 << seglog)
                          ? tile_bits(pr, bp, which, (uint64_t(r) << logS) + c0 + sg * SEG)
                          : 0u;
        }
        if (!built) {
            p1tw_build<F>(tb, tfwd, c0, SEG, seglog, logR1, logN);
            built = true;
        }
#pragma unroll
        for (int u = 0; u < kLoadBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= (R1 << seglog)) break;
            const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
            T x[SEG];
#pragma unroll
            for (int c = 0; c < SEG; ++c) x[c] = (bits[u] >> c) & 1u;
            seg_store<T>(sm + lay.at(r, sg * SEG), x);
        }
    }
    if (!built) p1tw_build<F>(tb, tfwd, c0, SEG, seglog, logR1, logN);
    __syncthreads();
    dif_columns<F, true>(sm, lay, logR1, logC, st);
    const int per = 32 + (1 << (logR1 - 5));
    const T *tc = tb + (per << seglog);
    const int nseg = R1 << seglog;
    // kTwBatch segments per thread at once, so their product chains overlap
    for (int e0 = threadIdx.x; e0 < nseg; e0 += kTwBatch * blockDim.x) {
#pragma unroll
        for (int u = 0; u < kTwBatch; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e < nseg) {
                const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
                T x[SEG];
                seg_load<T>(x, sm + lay.at(r, sg * SEG));
                const uint32_t f = __brev(static_cast<uint32_t>(r)) >> (32 - logR1);
                const T *ta = tb + sg * per;
                const T base = F::mul_full(ta[f & 31], ta[32 + (f >> 5)]);  // w^(t0 f), full form
                const T step = F::mul_full(tc[f & 31], tc[32 + (f >> 5)]);  // w^f, full form
                twiddle_segment<F, SEG>(x, base, step);
                stcg256(dst + (uint64_t(r) << logS) + c0 + sg * SEG, x);
            }
        }
    }
    __syncthreads();
    (void)C;
}

// Pass 2 of both spectra (rows of R2 = 2^logR2, C2 rows from row group rg), the pointwise
// product and the inverse pass 2; X = key spectrum, W = window spectrum.
template <class F>
__device__ __forceinline__ void body_fused_last(typename F::T *sm, const typename F::Tw *stf,
                                const typename F::Tw *sti, uint64_t rg, int logR2, int logC,
                                typename F::T *__restrict__ X, typename F::T *__restrict__ W) {
    using T = typename F::T;
    const int C = 1 << logC;
    constexpr int V = 16 / sizeof(T);  // elements per 16-byte vector
    const int R2 = 1 << logR2;
    const uint64_t base = (rg << logC) << logR2;
    const auto lay = PassLay<T>::make(logR2);
    const int cnt = R2 << logC;
    if constexpr (sizeof(T) == 4) {
        stage_rows(sm, lay, 0, X + base, cnt, logR2);
        stage_rows(sm, lay, C, W + base, cnt, logR2);
        cp_async_wait_all();
    } else {
        for (int e = threadIdx.x * V; e < cnt; e += blockDim.x * V) {
            const int c = e >> logR2, r = e & (R2 - 1);
            const uint4 xv = __ldcg(reinterpret_cast<const uint4 *>(X + base + e));
            const uint4 wv = __ldcg(reinterpret_cast<const uint4 *>(W + base + e));
            const T *xs = reinterpret_cast<const T *>(&xv), *ws = reinterpret_cast<const T *>(&wv);
#pragma unroll
            for (int k = 0; k < V; ++k) {
                sm[lay.at(r + k, c)] = xs[k];
                sm[lay.at(r + k, C + c)] = ws[k];
            }
        }
    }
    __syncthreads();
    // logR2 >= 6 for every two-pass transform (N >= 2^13)
    product_columns<F>(sm, lay, logR2, logC, stf, sti, [](T a, T b) { return F::mont(a, b); });
    store_rows(W + base, sm, lay, C, cnt, logR2);
    __syncthreads();
}

// Inverse pass 1 on column group cg of the product, scale, low bit, XOR output bits.
template <class F>
__device__ __forceinline__ void body_inv_first(typename F::T *sm, const typename F::Tw *st, const TilePair &pr,
                               const BlockPtrs &bp, uint64_t cg, int logN, int logR1, int logC,
                               const typename F::T *__restrict__ src,
                               const typename F::Tw *__restrict__ tinv, typename F::Tw scale) {
    using T = typename F::T;
    constexpr int SEG = 32 / sizeof(T), logSEG = sizeof(T) == 4 ? 3 : 2;
    const int R1 = 1 << logR1, logS = logN - logR1;
    const uint64_t c0 = cg << logC;
    const RowMajor lay{logC};
    const int seglog = logC - logSEG;
    // the inverse twiddles w^-(t f) from short tables (p1tw_build with the inverse roots),
    // looked up while the rows load, applied in one pass over shared memory
    T *tb = sm + (R1 << logC);
    {
        // the two 16-byte halves of a row segment come from two adjacent lanes (a warp's
        // copy reads 16 whole sectors)
        for (int e = threadIdx.x; e < 2 * (R1 << seglog); e += blockDim.x) {
            const int si = e >> 1, h = e & 1;
            const int r = si >> seglog, sg = si & ((1 << seglog) - 1);
            const uint4 *g = reinterpret_cast<const uint4 *>(src + (uint64_t(r) << logS) + c0 + sg * SEG);
            uint4 *d = reinterpret_cast<uint4 *>(sm + lay.at(r, sg * SEG));
            cp_async16(d + h, g + h);
        }
        p1tw_build<F>(tb, tinv, c0, SEG, seglog, logR1, logN);
        cp_async_wait_all();
    }
    __syncthreads();
    {
        const int per = 32 + (1 << (logR1 - 5));
        const T *tc = tb + (per << seglog);
        const int nseg = R1 << seglog;
        for (int e0 = threadIdx.x; e0 < nseg; e0 += kTwBatch * blockDim.x) {
#pragma unroll
            for (int u = 0; u < kTwBatch; ++u) {
                const int e = e0 + u * blockDim.x;
                if (e < nseg) {
                    const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
                    T x[SEG];
                    seg_load<T>(x, sm + lay.at(r, sg * SEG));
                    const uint32_t f = __brev(static_cast<uint32_t>(r)) >> (32 - logR1);
                    const T *ta = tb + sg * per;
                    const T base = F::mul_full(ta[f & 31], ta[32 + (f >> 5)]);
                    const T step = F::mul_full(tc[f & 31], tc[32 + (f >> 5)]);
                    twiddle_segment<F, SEG>(x, base, step);
                    seg_store<T>(sm + lay.at(r, sg * SEG), x);
                }
            }
        }
    }
    __syncthreads();
    dit_columns<F, true>(sm, lay, logR1, logC, st);
    // segment (r, sg) holds conv indices k = r*S1 + c0 + sg*SEG + c: SEG output bits
    for (int e = threadIdx.x; e < (R1 << seglog); e += blockDim.x) {
        const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
        const uint64_t k0 = (uint64_t(r) << logS) + c0 + sg * SEG;
        if (k0 + SEG <= pr.K0 || k0 >= uint64_t(pr.K0) + pr.out_len) continue;
        T x[SEG];
        seg_load<T>(x, sm + lay.at(r, sg * SEG));
        uint32_t byte = 0;
#pragma unroll
        for (int c = 0; c < SEG; ++c) {
            const uint64_t k = k0 + c;
            if (k >= pr.K0 && k < uint64_t(pr.K0) + pr.out_len)
                byte |= F::low_bit(F::mul_tw(x[c], scale)) << c;
        }
        if (byte) {
            const uint64_t pos = pr.out_bit0 + (k0 - pr.K0);  // multiple of SEG
            atomicXor(bp.out32 + (pos >> 5), byte << (pos & 31));
        }
    }
    __syncthreads();
}

// Forward pass 2 of one fd spectrum in place: C = 2^logC rows of R2 = 2^logR2 from row
// group rg.
template <class F>
__device__ __forceinline__ void body_fwd_last(typename F::T *sm, const typename F::Tw *stf, uint64_t rg, int logR2,
                              int logC, typename F::T *__restrict__ A) {
    using T = typename F::T;
    constexpr int V = 16 / sizeof(T);
    const int R2 = 1 << logR2;
    const uint64_t base = (rg << logC) << logR2;
    const auto lay = PassLay<T>::make(logR2);
    const int cnt = R2 << logC;
    if constexpr (sizeof(T) == 4) {
        stage_rows(sm, lay, 0, A + base, cnt, logR2);
        cp_async_wait_all();
    } else {
        for (int e = threadIdx.x * V; e < cnt; e += blockDim.x * V) {
            const int c = e >> logR2, r = e & (R2 - 1);
            const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(A + base + e));
            const T *xs = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int k = 0; k < V; ++k) sm[lay.at(r + k, c)] = xs[k];
        }
    }
    __syncthreads();
    dif_columns<F, false>(sm, lay, logR2, logC, stf);
    store_rows(A + base, sm, lay, 0, cnt, logR2);
    __syncthreads();
}

// Rows of up to kSum4Out output tiles I0 .. I0+nout-1 from row group rg (E = max(2048, R2)
// elements of each): Z_I = sum over the key tiles J in [jlo, jhi) of X_J * W_{wmap[I][J]}
// (Montgomery products summed in the field; Q key tiles in all, the row length of the
// window-index table), then the inverse pass 2 of every row, written to Z_I
// (output tiles at stride N from Z). The sums run over chunks of 2048 elements, each
// accumulated in registers over all J and parked in shared memory, and each key-tile
// vector is loaded once for all the item's outputs. Shared memory: kSum4Out x C columns
// of R2 rows (C = 2048 / R2 rows per output, or one row when R2 > 2048).
constexpr int kSum4Elems = 2048;
template <class F>
__device__ __forceinline__ void body_sum4_inv_last(typename F::T *sm, const typename F::Tw *sti, uint64_t rg,
                                   int logR2, int logC, const typename F::T *__restrict__ X,
                                   const typename F::T *__restrict__ W,
                                   const uint32_t *__restrict__ wmap_blk, uint32_t Q, uint32_t jlo,
                                   uint32_t jhi, uint32_t I0,
                                   uint32_t nout, uint32_t consec, uint64_t N,
                                   typename F::T *__restrict__ Z) {
    using T = typename F::T;
    constexpr int V = 16 / sizeof(T);
    constexpr int VPT = kSum4Elems / (kThreads * V);  // vectors per thread: 1 (32-bit), 2 (64-bit)
    static_assert(VPT >= 1 && VPT * kThreads * V == kSum4Elems, "row-group size");
    static_assert(kSum4Out == 4, "the inverse pass runs on 4 C columns");
    const int R2 = 1 << logR2, C = 1 << logC;
    const int E = R2 << logC;  // elements of one output in this item
    const uint64_t base = (rg << logC) << logR2;
    const auto lay = PassLay<T>::make(logR2);
    for (int h0 = 0; h0 < E; h0 += kSum4Elems) {
        const uint64_t hb = base + h0;
        T acc[kSum4Out][VPT][V];
#pragma unroll
        for (int o = 0; o < kSum4Out; ++o)
#pragma unroll
            for (int v = 0; v < VPT; ++v)
#pragma unroll
                for (int k = 0; k < V; ++k) acc[o][v][k] = 0;
        const auto vec = [&](const T *row, int v) {
            return __ldcg(reinterpret_cast<const uint4 *>(row + (threadIdx.x + v * kThreads) * V));
        };
        if (consec) {
            // window of (I0 + o, J) = d0 + o - J: the item's window rows slide by one per key
            // tile, so each J needs one new window row (output 0's) and the key-tile row;
            // both are loaded ahead (the key-tile row one step, the window row two steps)
            const int64_t d0 = static_cast<int64_t>(__ldg(wmap_blk)) + I0;
            uint4 wv[kSum4Out][VPT], xn[VPT], wn[VPT];
#pragma unroll
            for (int o = 0; o < kSum4Out; ++o)
#pragma unroll
                for (int v = 0; v < VPT; ++v)
                    wv[o][v] = o < static_cast<int>(nout)
                                   ? vec(W + uint64_t(d0 + o - int64_t(jlo)) * N + hb, v)
                                   : uint4{0, 0, 0, 0};
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                xn[v] = vec(X + uint64_t(jlo) * N + hb, v);
                wn[v] = jlo + 1 < jhi ? vec(W + uint64_t(d0 - int64_t(jlo) - 1) * N + hb, v)
                                      : uint4{0, 0, 0, 0};
            }
            for (uint32_t J = jlo; J < jhi; ++J) {
                uint4 xv[VPT];
#pragma unroll
                for (int v = 0; v < VPT; ++v) {
                    xv[v] = xn[v];
                    if (J + 1 < jhi) xn[v] = vec(X + uint64_t(J + 1) * N + hb, v);
                }
#pragma unroll
                for (int o = 0; o < kSum4Out; ++o)
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const T *xs = reinterpret_cast<const T *>(&xv[v]), *ws = reinterpret_cast<const T *>(&wv[o][v]);
#pragma unroll
                        for (int k = 0; k < V; ++k) acc[o][v][k] = F::add(acc[o][v][k], F::mont(xs[k], ws[k]));
                    }
                if (J + 1 < jhi) {
#pragma unroll
                    for (int o = kSum4Out - 1; o > 0; --o)
#pragma unroll
                        for (int v = 0; v < VPT; ++v) wv[o][v] = wv[o - 1][v];
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        wv[0][v] = wn[v];
                        if (J + 2 < jhi) wn[v] = vec(W + uint64_t(d0 - int64_t(J) - 2) * N + hb, v);
                    }
                }
            }
        } else {
            for (uint32_t J = jlo; J < jhi; ++J) {
                uint4 xv[VPT];
#pragma unroll
                for (int v = 0; v < VPT; ++v) xv[v] = vec(X + uint64_t(J) * N + hb, v);
#pragma unroll
                for (int o = 0; o < kSum4Out; ++o) {
                    if (o >= static_cast<int>(nout)) break;
                    const T *wj = W + uint64_t(__ldg(wmap_blk + uint64_t(I0 + o) * Q + J)) * N + hb;
#pragma unroll
                    for (int v = 0; v < VPT; ++v) {
                        const uint4 wv = vec(wj, v);
                        const T *xs = reinterpret_cast<const T *>(&xv[v]), *ws = reinterpret_cast<const T *>(&wv);
#pragma unroll
                        for (int k = 0; k < V; ++k) acc[o][v][k] = F::add(acc[o][v][k], F::mont(xs[k], ws[k]));
                    }
                }
            }
        }
        // output o's C rows are columns o C .. o C + C - 1 (the columns of outputs past nout
        // are transformed with the rest but never written)
#pragma unroll
        for (int o = 0; o < kSum4Out; ++o)
#pragma unroll
            for (int v = 0; v < VPT; ++v) {
                const int e = h0 + (threadIdx.x + v * kThreads) * V;
                const int c = e >> logR2, r = e & (R2 - 1);
                if constexpr (sizeof(T) == 4) {
                    *reinterpret_cast<uint4 *>(sm + lay.at(r, o * C + c)) =
                        make_uint4(acc[o][v][0], acc[o][v][1], acc[o][v][2], acc[o][v][3]);
                } else {
#pragma unroll
                    for (int k = 0; k < V; ++k) sm[lay.at(r + k, o * C + c)] = acc[o][v][k];
                }
            }
    }
    __syncthreads();
    dit_columns<F, false>(sm, lay, logR2, logC + 2, sti);
    for (int o = 0; o < static_cast<int>(nout); ++o) store_rows(Z + uint64_t(o) * N + base, sm, lay, o * C, E, logR2);
    __syncthreads();
}

// Streamed sum for a block with one output tile: for each key tile J, rows of row group
// rg of X_J and W_{wrow[J]} (after their forward pass 1) get the forward pass 2 in shared
// memory and their product is added to an accumulator; the accumulator then gets the
// inverse pass 2 and is written to Z. Shared memory: key, window and accumulator
// columns (3 C columns of R2 rows).
template <class F>
__device__ __forceinline__ void body_stream_sum(typename F::T *sm, const typename F::Tw *stf,
                                const typename F::Tw *sti, uint64_t rg, int logR2, int logC,
                                const typename F::T *__restrict__ X,
                                const typename F::T *__restrict__ W,
                                const uint32_t *__restrict__ wrow, uint32_t Q, uint64_t N,
                                typename F::T *__restrict__ Z) {
    using T = typename F::T;
    constexpr int V = 16 / sizeof(T);
    const int C = 1 << logC;
    const int R2 = 1 << logR2;
    const uint64_t base = (rg << logC) << logR2;
    const auto lay = PassLay<T>::make(logR2);
    const int cnt = R2 << logC;
    T *acc = sm + 2 * C * lay.cs;
    // the window index of every key tile, fetched once (not one dependent load per tile)
    uint32_t *wix = reinterpret_cast<uint32_t *>(acc + C * lay.cs);
    for (int e = threadIdx.x; e < C * lay.cs; e += blockDim.x) acc[e] = 0;
    for (uint32_t J = threadIdx.x; J < Q; J += blockDim.x) wix[J] = __ldg(wrow + J);
    __syncthreads();
    for (uint32_t J = 0; J < Q; ++J) {
        const T *xj = X + uint64_t(J) * N + base;
        const T *wj = W + uint64_t(wix[J]) * N + base;
        if constexpr (sizeof(T) == 4) {
            stage_rows(sm, lay, 0, xj, cnt, logR2);
            stage_rows(sm, lay, C, wj, cnt, logR2);
            cp_async_wait_all();
        } else {
            for (int e = threadIdx.x * V; e < cnt; e += blockDim.x * V) {
                const int c = e >> logR2, r = e & (R2 - 1);
                const uint4 xv = __ldcg(reinterpret_cast<const uint4 *>(xj + e));
                const uint4 wv = __ldcg(reinterpret_cast<const uint4 *>(wj + e));
                const T *xs = reinterpret_cast<const T *>(&xv), *ws = reinterpret_cast<const T *>(&wv);
#pragma unroll
                for (int k = 0; k < V; ++k) {
                    sm[lay.at(r + k, c)] = xs[k];
                    sm[lay.at(r + k, C + c)] = ws[k];
                }
            }
        }
        __syncthreads();
        product_acc_columns<F>(sm, lay, logR2, logC, 2 * C, stf,
                               [](T a, T b) { return F::mont(a, b); },
                               [](T a, T b) { return F::add(a, b); });
    }
    dit_columns<F, false>(acc, lay, logR2, logC, sti);
    store_rows(Z + base, acc, lay, 0, cnt, logR2);
    __syncthreads();
}

// Outer convolution for bins [k0, k0 + C) of one sum group and output slice: with
// A_t = X_{jlo+t}[k] (t < Qg) and B_u = W_{wb+u}[k] (u < Ps + Qg - 1), the slice's sums are
// Z_{out+i}[k] = sum_t A_t B_{i-t+Qg-1} = (A * B)[i + Qg - 1], taken from a cyclic
// convolution of T >= Ps + Qg - 1 points over the tile index (outputs Qg - 1 .. Qg + Ps - 2
// are unaliased), scaled by 1/T: the same field values the direct sums give. Shared memory:
// the forward tile (T rows of [A_t | B_t], 2C columns), the product tile (T rows of C).
// When log2 T = 1 mod 4 (a one-stage round in the usual split), the forward transform's first
// stage (rows r, r + T/2) runs on the rows as they are loaded and the inverse's last stage
// only on the Ps rows written out, so that no round is that short.
template <class F>
__device__ __forceinline__ void body_outer(typename F::T *sm, const typename F::Tw *stf, const typename F::Tw *sti,
                           uint64_t k0, int logT, int logCo, uint32_t Qg, uint32_t Ps,
                           const typename F::T *__restrict__ X, const typename F::T *__restrict__ W,
                           typename F::T *__restrict__ Z, uint64_t N, typename F::Tw tinv) {
    using T = typename F::T;
    using Tw = typename F::Tw;
    constexpr int V = 16 / sizeof(T);
    const int R = 1 << logT, C = 1 << logCo, H = R >> 1;
    const RowMajor lay2{logCo + 1}, lay{logCo};
    T *fw = sm, *pr = sm + (R << (logCo + 1));
    const uint32_t nb = Ps + Qg - 1;
    const int vpr = C / V;  // 16-byte pieces per operand row
    const bool fuse = (logT & 3) == 1;
    const int units = 2 * H * vpr;
    if (!fuse) {
        for (int e = threadIdx.x; e < 2 * R * vpr; e += blockDim.x) {
            const int r = e / (2 * vpr), q = e - r * 2 * vpr;
            const int which = q >= vpr, v = which ? q - vpr : q;
            T *dst = fw + lay2.at(r, which * C + v * V);
            if (which ? uint32_t(r) < nb : uint32_t(r) < Qg)
                cp_async16(dst, (which ? W : X) + uint64_t(r) * N + k0 + v * V);
            else
                *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
        }
        cp_async_wait_all();
    }
    // fused: two (row pair, piece) units per thread at a time, their four loads issued together
    for (int e0 = threadIdx.x; fuse && e0 < units; e0 += 2 * blockDim.x) {
        uint4 lo[2], hi[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = e0 + u * blockDim.x;
            lo[u] = hi[u] = make_uint4(0u, 0u, 0u, 0u);
            if (e < units) {
                const int r = e / (2 * vpr), q = e - r * 2 * vpr;
                const int which = q >= vpr, v = which ? q - vpr : q;
                const uint32_t lim = which ? nb : Qg;
                const T *src = (which ? W : X) + k0 + v * V;
                if (uint32_t(r) < lim) lo[u] = __ldcg(reinterpret_cast<const uint4 *>(src + uint64_t(r) * N));
                if (uint32_t(r + H) < lim)
                    hi[u] = __ldcg(reinterpret_cast<const uint4 *>(src + uint64_t(r + H) * N));
            }
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int e = e0 + u * blockDim.x;
            if (e >= units) break;
            const int r = e / (2 * vpr), q = e - r * 2 * vpr;
            const int col = (q >= vpr ? C : 0) + (q >= vpr ? q - vpr : q) * V;
            T *a = reinterpret_cast<T *>(&lo[u]), *b = reinterpret_cast<T *>(&hi[u]);
            const Tw w = stf[H - 1 + r];
#pragma unroll
            for (int k = 0; k < V; ++k) F::dif_bfly(a[k], b[k], w);
            *reinterpret_cast<uint4 *>(fw + lay2.at(r, col)) = lo[u];
            *reinterpret_cast<uint4 *>(fw + lay2.at(r + H, col)) = hi[u];
        }
    }
    __syncthreads();
    if (fuse)
        dif_columns_after_first<F, true>(fw, lay2, logT, logCo + 1, stf);
    else
        dif_columns<F, true>(fw, lay2, logT, logCo + 1, stf);
    for (int e = threadIdx.x; e < (R << logCo); e += blockDim.x) {
        const int r = e >> logCo, c = e & (C - 1);
        pr[lay.at(r, c)] = F::mont(fw[lay2.at(r, c)], fw[lay2.at(r, C + c)]);
    }
    __syncthreads();
    if (!fuse) {
        dit_columns<F, true>(pr, lay, logT, logCo, sti);
        for (int e = threadIdx.x; e < int(Ps) * vpr; e += blockDim.x) {
            const int i = e / vpr, v = e - i * vpr;
            const T *src = pr + lay.at(i + int(Qg) - 1, v * V);
            T o[V];
#pragma unroll
            for (int k = 0; k < V; ++k) o[k] = F::mul_tw(src[k], tinv);
            __stcg(reinterpret_cast<uint4 *>(Z + uint64_t(i) * N + k0 + v * V), *reinterpret_cast<uint4 *>(o));
        }
        __syncthreads();
        return;
    }
    dit_columns_but_last<F, true>(pr, lay, logT, logCo, sti);
    for (int e = threadIdx.x; e < int(Ps) * vpr; e += blockDim.x) {
        const int i = e / vpr, v = e - i * vpr;
        const int y = i + int(Qg) - 1, j = y & (H - 1);
        const T *pa = pr + lay.at(j, v * V), *pb = pr + lay.at(j + H, v * V);
        const Tw w = sti[H - 1 + j];
        T o[V];
#pragma unroll
        for (int k = 0; k < V; ++k) {
            T a = pa[k], b = pb[k];
            F::dit_bfly(a, b, w);
            o[k] = F::mul_tw(y < H ? a : b, tinv);
        }
        __stcg(reinterpret_cast<uint4 *>(Z + uint64_t(i) * N + k0 + v * V), *reinterpret_cast<uint4 *>(o));
    }
    __syncthreads();
}

// Inverse pass 2 of one fd output spectrum in place: C = 2^logC rows of R2 = 2^logR2 from
// row group rg (the mirror of body_fwd_last).
template <class F>
__device__ __forceinline__ void body_inv_last(typename F::T *sm, const typename F::Tw *sti, uint64_t rg, int logR2,
                              int logC, typename F::T *__restrict__ A) {
    using T = typename F::T;
    constexpr int V = 16 / sizeof(T);
    const int R2 = 1 << logR2;
    const uint64_t base = (rg << logC) << logR2;
    const auto lay = PassLay<T>::make(logR2);
    const int cnt = R2 << logC;
    if constexpr (sizeof(T) == 4) {
        stage_rows(sm, lay, 0, A + base, cnt, logR2);
        cp_async_wait_all();
    } else {
        for (int e = threadIdx.x * V; e < cnt; e += blockDim.x * V) {
            const int c = e >> logR2, r = e & (R2 - 1);
            const uint4 v = __ldcg(reinterpret_cast<const uint4 *>(A + base + e));
            const T *xs = reinterpret_cast<const T *>(&v);
#pragma unroll
            for (int k = 0; k < V; ++k) sm[lay.at(r + k, c)] = xs[k];
        }
    }
    __syncthreads();
    dit_columns<F, false>(sm, lay, logR2, logC, sti);
    store_rows(A + base, sm, lay, 0, cnt, logR2);
    __syncthreads();
}

// ---------------------------------------------------------------- the persistent kernel
//
// CTAs pull items from the list with an atomic counter; the list is ordered so that
// each item depends only on items before it, which are already claimed by running
// CTAs, so every wait ends. Waits are bounded anyway: on timeout the status word gets
// PA_ERR_TIMEOUT and the item's body is skipped.
// Counters: c1/c2/c3 per tile (pass 1, 2, 3 items done), then the list position, then
// per fd block the forward pass-2 items done, then per fd block the forward pass-1 items
// done.

template <class F>
__global__ void __launch_bounds__(kThreads, kMinBlocks<F>) ntt_persistent(
    const uint64_t *__restrict__ items, uint32_t nitems, const NttTile *__restrict__ tiles,
    const FdBlock *__restrict__ fds, const uint32_t *__restrict__ wmap,
    const BlockPtrs *__restrict__ blks, BlockPtrs one, typename F::T *__restrict__ ws,
    const typename F::Tw *__restrict__ stage, const typename F::Tw *__restrict__ tfwd,
    const typename F::Tw *__restrict__ tinv, uint32_t *cnt, uint32_t ntiles, uint32_t nfd,
    uint32_t slots, int *status) {
    using T = typename F::T;
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint64_t cur;
    __shared__ int flag;
    // Stage tables stay in shared memory across items: slot 0 at st0 and slot 1 right
    // after it hold (direction, log2 R) = skey[slot] (-1: nothing valid). A body whose tile
    // starts right after slot 0 overwrites slot 1.
    __shared__ int skey[2];
    if (threadIdx.x == 0) skey[0] = skey[1] = -1;
    uint32_t *c1 = cnt, *c2 = cnt + ntiles, *c3 = cnt + 2 * uint64_t(ntiles);
    uint32_t *next = cnt + 3 * uint64_t(ntiles), *cfd = next + 1, *cfd1 = cfd + nfd;
    Tw *st0 = reinterpret_cast<Tw *>(smraw);
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t i = atomicAdd(next, 1u);
            cur = i < nitems ? items[i] : ~0ull;
        }
        __syncthreads();
        const uint64_t it = cur;
        const int k0 = skey[0], k1 = skey[1];
        __syncthreads();
        if (it == ~0ull) break;
        const uint32_t type = static_cast<uint32_t>(it >> 60);
        const uint32_t ti = static_cast<uint32_t>((it >> 32) & 0x0FFFFFFFu);
        const uint32_t sub = static_cast<uint32_t>(it);
        const NttTile tl = tiles[ti];
        const BlockPtrs bp = pick(blks, one, tl.p.blk);
        Tw scale;
        memcpy(&scale, &tl.scale, sizeof(Tw));
        const int logN = static_cast<int>(tl.logN);
        const int logR1 = static_cast<int>(tl.logR1), logR2 = static_cast<int>(tl.logR2);
        const int logC1 = static_cast<int>(tl.logC1), logC2 = static_cast<int>(tl.logC2);
        T *X = ws + tl.ws_off;
        T *W = X + (uint64_t(1) << logN);
        switch (type) {
            case IT_SMALL: {
                Tw *sti = st0 + (1 << logN);
                if (k0 != logN) load_stage<F>(st0, stage, 0, logN);
                if (k0 != logN || k1 != 32 + logN) load_stage<F>(sti, stage, 1, logN);
                body_small<F>(reinterpret_cast<T *>(sti + (1 << logN)), st0, sti, tl.p, bp, logN, scale);
                break;
            }
            case IT_P1: {
                // the spectra slot is reused: wait until the tile `slots` earlier released it
                bool ok = true;
                if (ti >= slots) ok = wait_count(c3 + (ti - slots), tiles[ti - slots].g1, status, &flag);
                const int which = sub >= tl.g1 ? 1 : 0;
                if (k0 != logR1) load_stage<F>(st0, stage, 0, logR1);
                if (ok)
                    body_fwd_first<F>(reinterpret_cast<T *>(st0 + (1 << logR1)), st0, tl.p, bp, which,
                                      sub - which * tl.g1, logN, logR1, logC1, which ? W : X, tfwd);
                signal_count(c1 + ti);
                break;
            }
            case IT_P2: {
                Tw *sti = st0 + (1 << logR2);
                if (k0 != logR2) load_stage<F>(st0, stage, 0, logR2);
                if (k0 != logR2 || k1 != 32 + logR2) load_stage<F>(sti, stage, 1, logR2);
                if (wait_count(c1 + ti, 2 * tl.g1, status, &flag))
                    body_fused_last<F>(reinterpret_cast<T *>(sti + (1 << logR2)), st0, sti, sub, logR2,
                                       logC2, X, W);
                signal_count(c2 + ti);
                break;
            }
            case IT_P3: {
                if (k0 != 32 + logR1) load_stage<F>(st0, stage, 1, logR1);
                if (wait_count(c2 + ti, tl.g2, status, &flag))
                    body_inv_first<F>(reinterpret_cast<T *>(st0 + (1 << logR1)), st0, tl.p, bp, sub,
                                      logN, logR1, logC1, W, tinv, scale);
                signal_count(c3 + ti);
                break;
            }
            case IT_FD_P1: {
                if (k0 != logR1) load_stage<F>(st0, stage, 0, logR1);
                body_fwd_first<F>(reinterpret_cast<T *>(st0 + (1 << logR1)), st0, tl.p, bp,
                                  static_cast<int>(tl.which), sub, logN, logR1, logC1, X, tfwd);
                signal_count(c1 + ti);
                if (threadIdx.x == 0) atomicAdd(cfd1 + tl.fd, 1u);  // fenced by signal_count
                break;
            }
            case IT_FD_P2: {
                if (k0 != logR2) load_stage<F>(st0, stage, 0, logR2);
                if (wait_count(c1 + ti, tl.g1, status, &flag))
                    body_fwd_last<F>(reinterpret_cast<T *>(st0 + (1 << logR2)), st0, sub, logR2, logC2, X);
                signal_count(cfd + tl.fd);
                break;
            }
            case IT_FD_SUM: {  // output tiles tl.out .. + kSum4Out - 1 (sum tiles ti, ti + 1, ...)
                const FdBlock fb = fds[tl.fd];
                const uint32_t nout = min(static_cast<uint32_t>(kSum4Out), fb.P - tl.out);
                if (k0 != 32 + logR2) load_stage<F>(st0, stage, 1, logR2);
                if (wait_count(cfd + tl.fd, fb.nfwd2, status, &flag))
                    body_sum4_inv_last<F>(reinterpret_cast<T *>(st0 + (1 << logR2)), st0, sub, logR2,
                                          logC2, ws + fb.x_off, ws + fb.w_off, wmap + fb.wmap, fb.Q,
                                          tl.jlo, tl.jhi, tl.out, nout, fb.consec, uint64_t(1) << logN, X);
                signal_counts(c2 + ti, nout);
                break;
            }
            case IT_FD_STREAM: {
                const FdBlock fb = fds[tl.fd];
                Tw *sti = st0 + (1 << logR2);
                if (k0 != logR2) load_stage<F>(st0, stage, 0, logR2);
                if (k0 != logR2 || k1 != 32 + logR2) load_stage<F>(sti, stage, 1, logR2);
                if (wait_count(cfd1 + tl.fd, fb.nfwd1, status, &flag))
                    body_stream_sum<F>(reinterpret_cast<T *>(sti + (1 << logR2)), st0, sti, sub, logR2,
                                       logC2, ws + fb.x_off, ws + fb.w_off, wmap + fb.wmap, fb.Q,
                                       uint64_t(1) << logN, X);
                signal_count(c2 + ti);
                break;
            }
            case IT_FD_OUTER: {  // bins [sub 2^logCo, +2^logCo) of one sum group and slice
                const FdBlock fb = fds[tl.fd];
                const int logT = static_cast<int>(tl.logT);
                Tw *sti = st0 + (1 << logT);
                if (k0 != logT) load_stage<F>(st0, stage, 0, logT);
                if (k0 != logT || k1 != 32 + logT) load_stage<F>(sti, stage, 1, logT);
                if (wait_count(cfd + tl.fd, fb.nfwd2, status, &flag)) {
                    const uint64_t N = uint64_t(1) << logN;
                    body_outer<F>(reinterpret_cast<T *>(sti + (1 << logT)), st0, sti,
                                  uint64_t(sub) << tl.logCo, logT, static_cast<int>(tl.logCo),
                                  tl.jhi - tl.jlo, tl.nout, ws + fb.x_off + uint64_t(tl.jlo) * N,
                                  ws + fb.w_off + uint64_t(tl.wb) * N, X, N, scale);
                }
                signal_count(c1 + ti);
                break;
            }
            case IT_FD_INV2: {  // inverse pass 2 of sum tile ti, row group sub (after the outer items)
                if (k0 != 32 + logR2) load_stage<F>(st0, stage, 1, logR2);
                if (wait_count(c1 + tl.octr, tiles[tl.octr].g2, status, &flag))
                    body_inv_last<F>(reinterpret_cast<T *>(st0 + (1 << logR2)), st0, sub, logR2,
                                     logC2, X);
                signal_count(c2 + ti);
                break;
            }
            default: {  // IT_FD_P3
                if (k0 != 32 + logR1) load_stage<F>(st0, stage, 1, logR1);
                if (wait_count(c2 + ti, tl.g2, status, &flag))
                    body_inv_first<F>(reinterpret_cast<T *>(st0 + (1 << logR1)), st0, tl.p, bp, sub,
                                      logN, logR1, logC1, X, tinv, scale);
                __syncthreads();
                break;
            }
        }
        if (threadIdx.x == 0) {
            switch (type) {
                case IT_SMALL: skey[0] = logN; skey[1] = 32 + logN; break;
                case IT_P2:
                case IT_FD_STREAM: skey[0] = logR2; skey[1] = 32 + logR2; break;
                case IT_P1:
                case IT_FD_P1: skey[0] = logR1; skey[1] = -1; break;
                case IT_P3:
                case IT_FD_P3: skey[0] = 32 + logR1; skey[1] = -1; break;
                case IT_FD_P2: skey[0] = logR2; skey[1] = -1; break;
                case IT_FD_OUTER:
                    skey[0] = static_cast<int>(tl.logT);
                    skey[1] = 32 + static_cast<int>(tl.logT);
                    break;
                default: skey[0] = 32 + logR2; skey[1] = -1; break;  // IT_FD_SUM, IT_FD_INV2
            }
        }
    }
}

template <class F>
int launch_field(const NttLayout &lay, void *ws, const BlockPtrs *blks, const BlockPtrs &one,
                 int *status, Prof *prof, cudaStream_t s) {
    using Tw = typename F::Tw;
    Tables tab;
    int rc = ntt_tables(lay.field, &tab);
    if (rc != PA_OK) return rc;
    char *b = static_cast<char *>(ws);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(b + lay.off_counters);
    PA_CUDA_TRY(cudaMemsetAsync(cnt, 0, lay.counter_bytes, s));
    PA_CUDA_TRY(cudaFuncSetAttribute(ntt_persistent<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(lay.smem)));
    int per_sm = 0;
    PA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ntt_persistent<F>, kThreads,
                                                              lay.smem));
    int dev = 0, sms = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    PA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint64_t grid = uint64_t(per_sm > 0 ? per_sm : 1) * sms;
    if (grid > lay.nitems) grid = lay.nitems;
    prof_begin(prof, K_BATCH_PERSISTENT, s);
    ntt_persistent<F><<<static_cast<unsigned>(grid), kThreads, lay.smem, s>>>(
        reinterpret_cast<const uint64_t *>(b + lay.off_items), static_cast<uint32_t>(lay.nitems),
        reinterpret_cast<const NttTile *>(b + lay.off_tiles),
        reinterpret_cast<const FdBlock *>(b + lay.off_fd),
        reinterpret_cast<const uint32_t *>(b + lay.off_wmap), blks, one,
        reinterpret_cast<typename F::T *>(b + lay.off_spec), static_cast<const Tw *>(tab.stage),
        static_cast<const Tw *>(tab.fwd), static_cast<const Tw *>(tab.inv), cnt,
        static_cast<uint32_t>(lay.ntiles), static_cast<uint32_t>(lay.nfd), lay.slots, status);
    prof_end(prof, s);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace
}  // namespace pa
