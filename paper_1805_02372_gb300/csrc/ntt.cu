// Exact transform path: the tile products of the length-compatible decomposition
// (Sec. 3, Fig. 1-2, Steps 1-3) computed with number-theoretic transforms over a
// prime field instead of floating-point FFTs, so no rounding bound is needed.
//
// Decomposition. Output tile I covers rows [i0, i0+M), key tile J covers key bits
// [j0, j0+L) (L a multiple of 32, M of 64). With a[t] = x[j0+t] and the seed window
// w[u] = s[n-1+i0-j0-L+u] (positions outside the seed read as 0), output row i0+v
// receives coefficient L+v of the linear convolution a*w, and a cyclic convolution
// of size N >= L+M gives those coefficients unaliased. The tile's bits are XORed into
// the output (Eq. finalkey).
//
// Transforms. N = R1*R2 (a four-step split; R1, R2 <= 2^11) or N <= 2^12 in one CTA.
// Forward: decimation in frequency, natural input, bit-reversed spectrum; inverse:
// decimation in time from the bit-reversed spectrum, so no permutation pass exists.
// Each CTA does R-point transforms on columns in shared memory, two radix-2 stages
// per shared-memory round trip (radix-4 groups in registers).
//   ntt_fwd_first : pass 1 (stride R2) on the key tile and the seed window, read
//                   straight from the packed bits, then the four-step twiddles.
//   ntt_fused_last: pass 2 (contiguous rows of R2) of both spectra, the pointwise
//                   product, and inverse pass 2.
//   ntt_inv_first : twiddles, inverse pass 1, scale by N^-1, take bit 0, XOR the
//                   tile's output bytes into the packed output.
//   ntt_small     : N <= 2^12: all of the above in one CTA per tile.
#include <algorithm>
#include <mutex>
#include <stdio.h>
#include <string.h>
#include <vector>

#include "common.cuh"
#include "ntt_field.cuh"
#include "tiles.cuh"
#include "dft.cuh"

namespace pa {

constexpr int kLogMax = 22;           // largest transform: 2^22
constexpr int kLogSmallMax = 12;      // one-CTA transforms up to 2^12
constexpr int kThreads = 512;
// Two CTAs of 512 threads per SM for the 32-bit field (<= 64 registers), one for 64-bit.
template <class F>
constexpr int kMinBlocks = sizeof(typename F::T) == 4 ? 2 : 1;

// A transform tile of a batch: geometry plus its transform shape and spectra slot.
struct NttTile {
    TilePair p;
    uint64_t ws_off;  // element offset of the key spectrum (window spectrum follows)
    uint64_t scale;   // final scale as the bits of F::Tw
    uint32_t logN, logR1, logR2;
    uint32_t g1;      // pass-1 column groups (per input)
    uint32_t g2;      // pass-2 row groups
    uint32_t logC1;   // pass-1/3 columns per item (log2)
    uint32_t logC2;   // pass-2 rows per item (log2)
    uint32_t pad;
};

// Columns per pass-1/3 item and rows per pass-2 item (log2): at least one 32-byte row
// segment, and enough to give a 512-thread CTA about 8192 (32-bit) elements per item.
inline void pass_columns(int logN, size_t elem, int *logC1, int *logC2) {
    const int logR1 = (logN + 1) / 2, logR2 = logN / 2, logS = logN - logR1;
    const int target = elem == 4 ? 13 : 12;
    int c1 = std::max(elem == 4 ? 3 : 2, target - logR1);
    int c2 = std::max(elem == 4 ? 2 : 1, target - logR2);
    *logC1 = std::min(c1, logS);
    *logC2 = std::min(c2, logR1);
}

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
struct Tables {
    void *fwd = nullptr, *inv = nullptr;
    void *stage = nullptr;  // compact stage tables, see stage_table()
};
constexpr int kStageBlock = 4096;  // entries per (direction, log2 R) block
std::mutex g_tab_mu;
Tables g_tabs[2][64];

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
__device__ void body_small(typename F::T *sm, const typename F::Tw *stf, const typename F::Tw *sti,
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

// Row r of a pass-1 column group holds frequency f = brev(r); its C columns t = c0 + c
// need the twiddles w_N^(t f): w_N^(c0 f) from the table, then powers of w_N^f.
template <class F, int C>
__device__ __forceinline__ void row_twiddle(typename F::T (&x)[C], const typename F::Tw *tab,
                                            uint64_t c0, uint32_t f, int logN) {
    const int sh = kLogMax - logN;
    const typename F::Tw w0 = tw_at<F>(tab, static_cast<uint32_t>((c0 * f) << sh));
    const typename F::Tw step = tw_at<F>(tab, f << sh);
    typename F::T wf = F::full_form(w0);
    x[0] = F::mul_tw(x[0], w0);
#pragma unroll
    for (int c = 1; c < C; ++c) {
        wf = F::step_full(wf, step);
        x[c] = F::mul_full(x[c], wf);
    }
}

// Pass 1 forward on column group cg (C = 2^logC columns at stride S1 = N / R1); each
// thread handles 32-byte row segments (SEG columns).
template <class F>
__device__ void body_fwd_first(typename F::T *sm, const typename F::Tw *st, const TilePair &pr,
                               const BlockPtrs &bp, int which, uint64_t cg, int logN, int logR1,
                               int logC, typename F::T *__restrict__ dst,
                               const typename F::Tw *__restrict__ tfwd) {
    using T = typename F::T;
    constexpr int SEG = 32 / sizeof(T), logSEG = sizeof(T) == 4 ? 3 : 2;
    const int R1 = 1 << logR1, logS = logN - logR1, C = 1 << logC;
    const uint64_t c0 = cg << logC;
    const RowMajor lay{logC};
    const int seglog = logC - logSEG;  // segments per row (log2)
    for (int e = threadIdx.x; e < (R1 << seglog); e += blockDim.x) {
        const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
        const uint32_t bits = tile_bits(pr, bp, which, (uint64_t(r) << logS) + c0 + sg * SEG);
#pragma unroll
        for (int c = 0; c < SEG; ++c) sm[lay.at(r, sg * SEG + c)] = (bits >> c) & 1u;
    }
    __syncthreads();
    dif_columns<F, true>(sm, lay, logR1, logC, st);
    for (int e = threadIdx.x; e < (R1 << seglog); e += blockDim.x) {
        const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
        T x[SEG];
        const uint4 *src = reinterpret_cast<const uint4 *>(sm + lay.at(r, sg * SEG));
        *reinterpret_cast<uint4 *>(&x[0]) = src[0];
        *reinterpret_cast<uint4 *>(&x[SEG / 2]) = src[1];
        row_twiddle<F, SEG>(x, tfwd, c0 + sg * SEG, __brev(static_cast<uint32_t>(r)) >> (32 - logR1),
                            logN);
        uint4 *d = reinterpret_cast<uint4 *>(dst + (uint64_t(r) << logS) + c0 + sg * SEG);
        __stcg(d, *reinterpret_cast<uint4 *>(&x[0]));
        __stcg(d + 1, *reinterpret_cast<uint4 *>(&x[SEG / 2]));
    }
    __syncthreads();
    (void)C;
}

// Pass 2 of both spectra (rows of R2 = 2^logR2, C2 rows from row group rg), the pointwise
// product and the inverse pass 2; X = key spectrum, W = window spectrum.
template <class F>
__device__ void body_fused_last(typename F::T *sm, const typename F::Tw *stf,
                                const typename F::Tw *sti, uint64_t rg, int logR2, int logC,
                                typename F::T *__restrict__ X, typename F::T *__restrict__ W) {
    using T = typename F::T;
    const int C = 1 << logC;
    constexpr int V = 16 / sizeof(T);  // elements per 16-byte vector
    const int R2 = 1 << logR2;
    const uint64_t base = (rg << logC) << logR2;
    const ColMajor lay{ColMajor::stride(R2)};
    const int cnt = R2 << logC;
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
    __syncthreads();
    // logR2 >= 6 for every two-pass transform (N >= 2^13)
    dif_columns_head<F, false>(sm, lay, logR2, logC + 1, stf);
    product_round<F>(sm, lay, logR2, logC, stf, sti, [](T a, T b) { return F::mont(a, b); });
    dit_columns_tail<F, false>(sm + C * lay.cs, lay, logR2, logC, sti);
    for (int e = threadIdx.x * V; e < cnt; e += blockDim.x * V) {
        const int c = e >> logR2, r = e & (R2 - 1);
        uint4 ov;
        T *os = reinterpret_cast<T *>(&ov);
#pragma unroll
        for (int k = 0; k < V; ++k) os[k] = sm[lay.at(r + k, C + c)];
        __stcg(reinterpret_cast<uint4 *>(W + base + e), ov);
    }
    __syncthreads();
}

// Inverse pass 1 on column group cg of the product, scale, low bit, XOR output bits.
template <class F>
__device__ void body_inv_first(typename F::T *sm, const typename F::Tw *st, const TilePair &pr,
                               const BlockPtrs &bp, uint64_t cg, int logN, int logR1, int logC,
                               const typename F::T *__restrict__ src,
                               const typename F::Tw *__restrict__ tinv, typename F::Tw scale) {
    using T = typename F::T;
    constexpr int SEG = 32 / sizeof(T), logSEG = sizeof(T) == 4 ? 3 : 2;
    const int R1 = 1 << logR1, logS = logN - logR1;
    const uint64_t c0 = cg << logC;
    const RowMajor lay{logC};
    const int seglog = logC - logSEG;
    for (int e = threadIdx.x; e < (R1 << seglog); e += blockDim.x) {
        const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
        T x[SEG];
        const uint4 *g = reinterpret_cast<const uint4 *>(src + (uint64_t(r) << logS) + c0 + sg * SEG);
        *reinterpret_cast<uint4 *>(&x[0]) = __ldcg(g);
        *reinterpret_cast<uint4 *>(&x[SEG / 2]) = __ldcg(g + 1);
        row_twiddle<F, SEG>(x, tinv, c0 + sg * SEG, __brev(static_cast<uint32_t>(r)) >> (32 - logR1),
                            logN);
        uint4 *d = reinterpret_cast<uint4 *>(sm + lay.at(r, sg * SEG));
        d[0] = *reinterpret_cast<uint4 *>(&x[0]);
        d[1] = *reinterpret_cast<uint4 *>(&x[SEG / 2]);
    }
    __syncthreads();
    dit_columns<F, true>(sm, lay, logR1, logC, st);
    // segment (r, sg) holds conv indices k = r*S1 + c0 + sg*SEG + c: SEG output bits
    for (int e = threadIdx.x; e < (R1 << seglog); e += blockDim.x) {
        const int r = e >> seglog, sg = e & ((1 << seglog) - 1);
        const uint64_t k0 = (uint64_t(r) << logS) + c0 + sg * SEG;
        if (k0 + SEG <= pr.K0 || k0 >= uint64_t(pr.K0) + pr.out_len) continue;
        uint32_t byte = 0;
#pragma unroll
        for (int c = 0; c < SEG; ++c) {
            const uint64_t k = k0 + c;
            if (k >= pr.K0 && k < uint64_t(pr.K0) + pr.out_len)
                byte |= F::low_bit(F::mul_tw(sm[lay.at(r, sg * SEG + c)], scale)) << c;
        }
        if (byte) {
            const uint64_t pos = pr.out_bit0 + (k0 - pr.K0);  // multiple of SEG
            atomicXor(bp.out32 + (pos >> 5), byte << (pos & 31));
        }
    }
    __syncthreads();
}

// ---------------------------------------------------------------- standalone kernels

template <class F>
__global__ void __launch_bounds__(kThreads, kMinBlocks<F>) ntt_small(const TilePair *__restrict__ pairs, BlockPtrs bp,
                                                      int logN,
                                                      const typename F::Tw *__restrict__ stage,
                                                      typename F::Tw scale) {
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smraw[];
    Tw *stf = reinterpret_cast<Tw *>(smraw);
    Tw *sti = stf + (1 << logN);
    const TilePair pr = pairs[blockIdx.x];
    load_stage<F>(stf, stage, 0, logN);
    load_stage<F>(sti, stage, 1, logN);
    body_small<F>(reinterpret_cast<typename F::T *>(sti + (1 << logN)), stf, sti, pr, bp, logN, scale);
}

template <class F>
__global__ void __launch_bounds__(kThreads, kMinBlocks<F>) ntt_fwd_first(const TilePair *__restrict__ pairs,
                                                          BlockPtrs bp, int logN, int logR1, int logC,
                                                          typename F::T *__restrict__ ws,
                                                          const typename F::Tw *__restrict__ stage,
                                                          const typename F::Tw *__restrict__ tfwd) {
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smraw[];
    Tw *st = reinterpret_cast<Tw *>(smraw);
    const int which = blockIdx.y & 1;
    const uint32_t pi = blockIdx.y >> 1;
    const TilePair pr = pairs[pi];
    typename F::T *dst = ws + (uint64_t(pi) * 2 + which) * (uint64_t(1) << logN);
    load_stage<F>(st, stage, 0, logR1);
    body_fwd_first<F>(reinterpret_cast<typename F::T *>(st + (1 << logR1)), st, pr, bp, which,
                      blockIdx.x, logN, logR1, logC, dst, tfwd);
}

template <class F>
__global__ void __launch_bounds__(kThreads, kMinBlocks<F>) ntt_fused_last(int logN, int logR2, int logC,
                                                           typename F::T *__restrict__ ws,
                                                           const typename F::Tw *__restrict__ stage) {
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smraw[];
    Tw *stf = reinterpret_cast<Tw *>(smraw);
    Tw *sti = stf + (1 << logR2);
    typename F::T *X = ws + (uint64_t(blockIdx.y) * 2) * (uint64_t(1) << logN);
    load_stage<F>(stf, stage, 0, logR2);
    load_stage<F>(sti, stage, 1, logR2);
    body_fused_last<F>(reinterpret_cast<typename F::T *>(sti + (1 << logR2)), stf, sti, blockIdx.x,
                       logR2, logC, X, X + (uint64_t(1) << logN));
}

template <class F>
__global__ void __launch_bounds__(kThreads, kMinBlocks<F>) ntt_inv_first(const TilePair *__restrict__ pairs,
                                                          BlockPtrs bp, int logN, int logR1, int logC,
                                                          const typename F::T *__restrict__ ws,
                                                          const typename F::Tw *__restrict__ stage,
                                                          const typename F::Tw *__restrict__ tinv,
                                                          typename F::Tw scale) {
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smraw[];
    Tw *st = reinterpret_cast<Tw *>(smraw);
    const uint32_t pi = blockIdx.y;
    const TilePair pr = pairs[pi];
    const typename F::T *src = ws + (uint64_t(pi) * 2 + 1) * (uint64_t(1) << logN);
    load_stage<F>(st, stage, 1, logR1);
    body_inv_first<F>(reinterpret_cast<typename F::T *>(st + (1 << logR1)), st, pr, bp, blockIdx.x,
                      logN, logR1, logC, src, tinv, scale);
}

// ---------------------------------------------------------------- persistent batched kernel
//
// One launch runs the transform tiles of every block of a batch. CTAs pull items from
// a work list with an atomic counter; the list is ordered so that each item depends
// only on items before it (pass 1 -> pass 2 -> pass 3 of the same tile), which are
// already claimed by running CTAs, so every wait ends. Waits are bounded anyway: on
// timeout the status word gets PA_ERR_TIMEOUT and the item is skipped.

template <class F>
__global__ void __launch_bounds__(kThreads, kMinBlocks<F>) ntt_persistent(
    const uint64_t *__restrict__ items, uint32_t nitems, const NttTile *__restrict__ tiles,
    const BlockPtrs *__restrict__ blks, typename F::T *__restrict__ ws,
    const typename F::Tw *__restrict__ stage, const typename F::Tw *__restrict__ tfwd,
    const typename F::Tw *__restrict__ tinv, uint32_t *c1, uint32_t *c2, uint32_t *c3,
    uint32_t slots, uint32_t *next, int *status) {
    using T = typename F::T;
    using Tw = typename F::Tw;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ uint64_t cur;
    __shared__ int flag;
    Tw *st0 = reinterpret_cast<Tw *>(smraw);
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t i = atomicAdd(next, 1u);
            cur = i < nitems ? items[i] : ~0ull;
        }
        __syncthreads();
        const uint64_t it = cur;
        __syncthreads();
        if (it == ~0ull) break;
        const uint32_t type = static_cast<uint32_t>(it >> 62);
        const uint32_t ti = static_cast<uint32_t>((it >> 32) & 0x3FFFFFFFu);
        const uint32_t sub = static_cast<uint32_t>(it);
        const NttTile tl = tiles[ti];
        const BlockPtrs bp = blks[tl.p.blk];
        Tw scale;
        memcpy(&scale, &tl.scale, sizeof(Tw));
        const int logN = static_cast<int>(tl.logN);
        const int logR1 = static_cast<int>(tl.logR1), logR2 = static_cast<int>(tl.logR2);
        T *X = ws + tl.ws_off;
        T *W = X + (uint64_t(1) << logN);
        if (type == 0) {
            Tw *sti = st0 + (1 << logN);
            load_stage<F>(st0, stage, 0, logN);
            load_stage<F>(sti, stage, 1, logN);
            body_small<F>(reinterpret_cast<T *>(sti + (1 << logN)), st0, sti, tl.p, bp, logN, scale);
        } else if (type == 1) {
            // the spectra slot is reused: wait until the tile `slots` earlier released it
            bool ok = true;
            if (ti >= slots) ok = wait_count(c3 + (ti - slots), tiles[ti - slots].g1, status, &flag);
            const int which = sub >= tl.g1 ? 1 : 0;
            load_stage<F>(st0, stage, 0, logR1);
            if (ok)
                body_fwd_first<F>(reinterpret_cast<T *>(st0 + (1 << logR1)), st0, tl.p, bp, which,
                                  sub - which * tl.g1, logN, logR1, static_cast<int>(tl.logC1),
                                  which ? W : X, tfwd);
            signal_count(c1 + ti);
        } else if (type == 2) {
            Tw *sti = st0 + (1 << logR2);
            load_stage<F>(st0, stage, 0, logR2);
            load_stage<F>(sti, stage, 1, logR2);
            if (wait_count(c1 + ti, 2 * tl.g1, status, &flag))
                body_fused_last<F>(reinterpret_cast<T *>(sti + (1 << logR2)), st0, sti, sub, logR2,
                                   static_cast<int>(tl.logC2), X, W);
            signal_count(c2 + ti);
        } else {
            load_stage<F>(st0, stage, 1, logR1);
            if (wait_count(c2 + ti, tl.g2, status, &flag))
                body_inv_first<F>(reinterpret_cast<T *>(st0 + (1 << logR1)), st0, tl.p, bp, sub,
                                  logN, logR1, static_cast<int>(tl.logC1), W, tinv, scale);
            signal_count(c3 + ti);
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- planning

namespace {

struct Geo {
    uint32_t logn;
    uint64_t L, M, pairs;
};

// Tile geometry for transform size 2^logn with output tile M: key tile L = N - M
// rounded down to 32 bits.
bool geo_for(uint64_t n, uint64_t m, uint32_t logn, uint64_t M, Geo *g) {
    const uint64_t N = uint64_t(1) << logn;
    if (M == 0 || M >= N) return false;
    uint64_t L = ((N - M) / 32) * 32;
    const uint64_t Lneed = round_up(n, 32);
    if (L > Lneed) L = Lneed;
    if (L == 0) return false;
    g->logn = logn;
    g->L = L;
    g->M = M;
    g->pairs = ceil_div(n, L) * ceil_div(m, M);
    return true;
}

}  // namespace

int ntt_plan(uint64_t n, uint64_t m, int path, const pa_opts *o, TransformCfg *c) {
    *c = TransformCfg();
    const int twoadic = path == PA_PATH_NTT31 ? F31::kTwoAdicity : F64::kTwoAdicity;
    (void)twoadic;
    if (path == PA_PATH_NTT31 && n >= F31::P) return PA_ERR_UNSUPPORTED;  // counts must stay < p
    Geo best{};
    double best_cost = 1e300;
    const uint32_t lo = 5, hi = kLogMax;
    const uint32_t force = o ? o->log2_transform : 0;
    const uint64_t Mforce = o ? o->tile_out : 0, Lforce = o ? o->tile_in : 0;
    for (uint32_t k = lo; k <= hi; ++k) {
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
            Geo g;
            uint64_t M = cands[i];
            if (M > round_up(m, 64)) M = round_up(m, 64);
            if (!geo_for(n, m, k, M, &g)) continue;
            if (Lforce) {
                const uint64_t L = round_up(Lforce, 32);
                if (L + M > N) continue;
                g.L = L;
                g.pairs = ceil_div(n, L) * ceil_div(m, M);
            }
            // cost ~ pairs * (3 transforms of N log N + fixed per-tile overhead)
            const double cost = double(g.pairs) * (double(N) * (k + 6) + 4096.0);
            if (cost < best_cost) {
                best_cost = cost;
                best = g;
            }
        }
    }
    if (best_cost >= 1e300) return PA_ERR_UNSUPPORTED;
    c->log2n = best.logn;
    c->L = best.L;
    c->M = best.M;
    c->tiles_in = ceil_div(n, best.L);
    c->tiles_out = ceil_div(m, best.M);
    if (best.logn <= kLogSmallMax) {
        c->passes = 1;
        c->radix_log2[0] = best.logn;
    } else {
        c->passes = 2;
        c->radix_log2[0] = (best.logn + 1) / 2;  // R1 (strided pass)
        c->radix_log2[1] = best.logn / 2;        // R2 (contiguous pass)
    }
    const uint64_t pairs = c->tiles_in * c->tiles_out;
    const size_t elem = path == PA_PATH_NTT31 ? 4 : 8;
    const uint64_t per_pair = c->passes == 1 ? 0 : 2 * (uint64_t(1) << best.logn) * elem;
    uint64_t conc = pairs;
    const uint64_t cap = uint64_t(2) << 30;  // 2 GiB of spectra per wave
    if (per_pair && conc * per_pair > cap) conc = cap / per_pair ? cap / per_pair : 1;
    if (conc > 65535 / 2) conc = 65535 / 2;
    c->concurrent = static_cast<uint32_t>(conc);
    return PA_OK;
}

size_t ntt_workspace(int path, const TransformCfg &c) {
    const size_t elem = path == PA_PATH_NTT31 ? 4 : 8;
    const uint64_t pairs = c.tiles_in * c.tiles_out;
    size_t bytes = round_up(pairs * sizeof(TilePair), 256);
    if (c.passes > 1) bytes += size_t(c.concurrent) * 2 * (size_t(1) << c.log2n) * elem;
    return bytes;
}

int ntt_init(const PlanCfg &cfg, void *ws) {
    std::vector<TilePair> pairs;
    make_pairs(cfg.n, cfg.m, cfg.tr, 0, &pairs);
    PA_CUDA_TRY(cudaMemcpy(ws, pairs.data(), pairs.size() * sizeof(TilePair), cudaMemcpyHostToDevice));
    Tables t;
    if (cfg.path == PA_PATH_NTT31) return get_tables<F31>(0, &t);
    return get_tables<F64>(1, &t);
}

namespace {

template <class F>
int launch_field(const PlanCfg &cfg, void *ws, Prof *prof, const uint64_t *seed, const uint64_t *key,
                 uint64_t *out, cudaStream_t s, int field) {
    using T = typename F::T;
    using Tw = typename F::Tw;
    Tables tab;
    int rc = get_tables<F>(field, &tab);
    if (rc != PA_OK) return rc;
    const TransformCfg &c = cfg.tr;
    const uint64_t npairs = c.tiles_in * c.tiles_out;
    const TilePair *pairs = static_cast<const TilePair *>(ws);
    T *spec = reinterpret_cast<T *>(static_cast<char *>(ws) + round_up(npairs * sizeof(TilePair), 256));
    BlockPtrs one{reinterpret_cast<const uint32_t *>(key), reinterpret_cast<const uint32_t *>(seed),
                  reinterpret_cast<uint32_t *>(out), cfg.n, cfg.m};
    const Tw *tf = static_cast<const Tw *>(tab.fwd), *ti = static_cast<const Tw *>(tab.inv);
    const Tw *stg = static_cast<const Tw *>(tab.stage);
    const Tw scale = FieldHost<F>::scale(c.log2n);
    const int logN = static_cast<int>(c.log2n);

    prof_begin(prof, K_MEMSET, s);
    PA_CUDA_TRY(cudaMemsetAsync(out, 0, ceil_div(cfg.m, 64) * 8, s));
    prof_end(prof, s);

    if (c.passes == 1) {
        const size_t smem = size_t(2) * (size_t(1) << logN) * sizeof(Tw) +
                            size_t(ColMajor::words(1 << logN, 2)) * sizeof(T);
        PA_CUDA_TRY(cudaFuncSetAttribute(ntt_small<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
        for (uint64_t p0 = 0; p0 < npairs; p0 += 65535) {
            const uint64_t cnt = npairs - p0 < 65535 ? npairs - p0 : 65535;
            prof_begin(prof, K_NTT_SMALL, s);
            ntt_small<F><<<static_cast<unsigned>(cnt), kThreads, smem, s>>>(pairs + p0, one, logN,
                                                                           stg, scale);
            prof_end(prof, s);
        }
        PA_CUDA_TRY(cudaGetLastError());
        return PA_OK;
    }
    const int logR1 = static_cast<int>(c.radix_log2[0]), logR2 = static_cast<int>(c.radix_log2[1]);
    int logC1 = 0, logC2 = 0;
    pass_columns(logN, sizeof(T), &logC1, &logC2);
    const size_t sm1 = (size_t(1) << logR1) * sizeof(Tw) + (size_t(1) << (logR1 + logC1)) * sizeof(T);
    const size_t sm2 = 2 * (size_t(1) << logR2) * sizeof(Tw) +
                       size_t(ColMajor::words(1 << logR2, 2 << logC2)) * sizeof(T);
    PA_CUDA_TRY(cudaFuncSetAttribute(ntt_fwd_first<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(sm1)));
    PA_CUDA_TRY(cudaFuncSetAttribute(ntt_inv_first<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(sm1)));
    PA_CUDA_TRY(cudaFuncSetAttribute(ntt_fused_last<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(sm2)));
    const unsigned gx1 = static_cast<unsigned>((uint64_t(1) << (logN - logR1)) >> logC1);
    const unsigned gx2 = static_cast<unsigned>((uint64_t(1) << logR1) >> logC2);
    for (uint64_t p0 = 0; p0 < npairs; p0 += c.concurrent) {
        const uint64_t cnt = npairs - p0 < c.concurrent ? npairs - p0 : c.concurrent;
        prof_begin(prof, K_NTT_FWD_FIRST, s);
        ntt_fwd_first<F><<<dim3(gx1, static_cast<unsigned>(2 * cnt)), kThreads, sm1, s>>>(
            pairs + p0, one, logN, logR1, logC1, spec, stg, tf);
        prof_end(prof, s);
        prof_begin(prof, K_NTT_FUSED_LAST, s);
        ntt_fused_last<F><<<dim3(gx2, static_cast<unsigned>(cnt)), kThreads, sm2, s>>>(
            logN, logR2, logC2, spec, stg);
        prof_end(prof, s);
        prof_begin(prof, K_NTT_INV_FIRST, s);
        ntt_inv_first<F><<<dim3(gx1, static_cast<unsigned>(cnt)), kThreads, sm1, s>>>(
            pairs + p0, one, logN, logR1, logC1, spec, stg, ti, scale);
        prof_end(prof, s);
    }
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace

// ---------------------------------------------------------------- batches

namespace {
size_t align256(size_t v) { return (v + 255) & ~size_t(255); }
}  // namespace

int ntt_batch_build(int path, const std::vector<BatchBlock> &blocks, uint32_t max_slots,
                    NttBatchInfo *info) {
    *info = NttBatchInfo();
    info->field = path == PA_PATH_NTT31 ? 0 : 1;
    const size_t elem = info->field == 0 ? 4 : 8, twsz = 8;
    std::vector<NttTile> big, small;
    for (const BatchBlock &b : blocks) {
        std::vector<TilePair> pairs;
        make_pairs(b.n, b.m, b.tr, b.index, &pairs);
        for (const TilePair &p : pairs) {
            NttTile t{};
            t.p = p;
            t.logN = b.tr.log2n;
            if (info->field == 0) {
                const F31::Tw sc = FieldHost<F31>::scale(t.logN);
                memcpy(&t.scale, &sc, sizeof(sc));
            } else {
                const F64::Tw sc = FieldHost<F64>::scale(t.logN);
                memcpy(&t.scale, &sc, sizeof(sc));
            }
            if (t.logN <= static_cast<uint32_t>(kLogSmallMax)) {
                small.push_back(t);
            } else {
                t.logR1 = (t.logN + 1) / 2;
                t.logR2 = t.logN / 2;
                int logC1 = 0, logC2 = 0;
                pass_columns(static_cast<int>(t.logN), elem, &logC1, &logC2);
                t.logC1 = static_cast<uint32_t>(logC1);
                t.logC2 = static_cast<uint32_t>(logC2);
                t.g1 = static_cast<uint32_t>((uint64_t(1) << (t.logN - t.logR1)) >> logC1);
                t.g2 = static_cast<uint32_t>((uint64_t(1) << t.logR1) >> logC2);
                big.push_back(t);
            }
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
    std::vector<NttTile> tiles = big;
    tiles.insert(tiles.end(), small.begin(), small.end());
    if (tiles.size() >= (size_t(1) << 30)) return PA_ERR_UNSUPPORTED;
    std::vector<uint64_t> items;
    auto push = [&items](uint64_t type, uint64_t ti, uint64_t sub) {
        items.push_back((type << 62) | (ti << 32) | sub);
    };
    // software pipeline: pass 1 of tile t, pass 2 of tile t-1, pass 3 of tile t-2
    const size_t nb = big.size();
    for (size_t t = 0; t < nb + 2; ++t) {
        if (t < nb)
            for (uint32_t k = 0; k < 2 * big[t].g1; ++k) push(1, t, k);
        if (t >= 1 && t - 1 < nb)
            for (uint32_t k = 0; k < big[t - 1].g2; ++k) push(2, t - 1, k);
        if (t >= 2 && t - 2 < nb)
            for (uint32_t k = 0; k < big[t - 2].g1; ++k) push(3, t - 2, k);
    }
    for (size_t i = 0; i < small.size(); ++i) push(0, nb + i, 0);
    if (items.size() >= (size_t(1) << 32)) return PA_ERR_UNSUPPORTED;
    info->ntiles = tiles.size();
    info->nitems = items.size();
    info->slots = static_cast<uint32_t>(slots ? slots : 1);
    // shared memory: the largest need among the bodies present
    size_t smem = 0;
    for (const NttTile &t : tiles) {
        if (t.logN <= static_cast<uint32_t>(kLogSmallMax)) {
            smem = std::max(smem, (size_t(2) << t.logN) * twsz +
                                      size_t(ColMajor::words(1 << t.logN, 2)) * elem);
        } else {
            const int logC1 = static_cast<int>(t.logC1), logC2 = static_cast<int>(t.logC2);
            smem = std::max(smem, (size_t(1) << t.logR1) * twsz + (size_t(1) << (t.logR1 + logC1)) * elem);
            smem = std::max(smem, 2 * (size_t(1) << t.logR2) * twsz +
                                      size_t(ColMajor::words(1 << t.logR2, 2 << logC2)) * elem);
        }
    }
    info->smem = smem;
    // workspace layout
    size_t off = 0;
    info->off_tiles = off;
    off = align256(off + tiles.size() * sizeof(NttTile));
    info->off_items = off;
    off = align256(off + items.size() * sizeof(uint64_t));
    info->off_counters = off;
    info->counter_bytes = (3 * tiles.size() + 1) * sizeof(uint32_t);
    off = align256(off + info->counter_bytes);
    info->off_spec = off;
    off = align256(off + size_t(info->slots) * slot_elems * elem);
    info->bytes = off;
    info->host_tiles.resize(tiles.size() * sizeof(NttTile));
    memcpy(info->host_tiles.data(), tiles.data(), info->host_tiles.size());
    info->host_items = items;
    return PA_OK;
}

int ntt_batch_upload(const NttBatchInfo &info, void *ws, cudaStream_t s) {
    char *b = static_cast<char *>(ws);
    if (!info.host_tiles.empty())
        PA_CUDA_TRY(cudaMemcpyAsync(b + info.off_tiles, info.host_tiles.data(),
                                    info.host_tiles.size(), cudaMemcpyHostToDevice, s));
    if (!info.host_items.empty())
        PA_CUDA_TRY(cudaMemcpyAsync(b + info.off_items, info.host_items.data(),
                                    info.host_items.size() * sizeof(uint64_t),
                                    cudaMemcpyHostToDevice, s));
    Tables t;
    return info.field == 0 ? get_tables<F31>(0, &t) : get_tables<F64>(1, &t);
}

namespace {
template <class F>
int batch_launch_field(const NttBatchInfo &info, void *ws, const void *blks, int *status, Prof *prof,
                       cudaStream_t s) {
    using Tw = typename F::Tw;
    Tables tab;
    int rc = get_tables<F>(info.field, &tab);
    if (rc != PA_OK) return rc;
    char *b = static_cast<char *>(ws);
    uint32_t *cnt = reinterpret_cast<uint32_t *>(b + info.off_counters);
    const uint32_t nt = static_cast<uint32_t>(info.ntiles);
    PA_CUDA_TRY(cudaMemsetAsync(cnt, 0, info.counter_bytes, s));
    PA_CUDA_TRY(cudaFuncSetAttribute(ntt_persistent<F>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(info.smem)));
    int per_sm = 0;
    PA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ntt_persistent<F>, kThreads,
                                                              info.smem));
    int dev = 0, sms = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    PA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint64_t grid = uint64_t(per_sm > 0 ? per_sm : 1) * sms;
    if (grid > info.nitems) grid = info.nitems;
    prof_begin(prof, K_BATCH_PERSISTENT, s);
    ntt_persistent<F><<<static_cast<unsigned>(grid), kThreads, info.smem, s>>>(
        reinterpret_cast<const uint64_t *>(b + info.off_items), static_cast<uint32_t>(info.nitems),
        reinterpret_cast<const NttTile *>(b + info.off_tiles), static_cast<const BlockPtrs *>(blks),
        reinterpret_cast<typename F::T *>(b + info.off_spec), static_cast<const Tw *>(tab.stage),
        static_cast<const Tw *>(tab.fwd), static_cast<const Tw *>(tab.inv), cnt, cnt + nt,
        cnt + 2 * nt, info.slots, cnt + 3 * nt, status);
    prof_end(prof, s);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}
}  // namespace

int ntt_batch_launch(const NttBatchInfo &info, void *ws, const void *blks, int *status, Prof *prof,
                     cudaStream_t s) {
    if (info.nitems == 0) return PA_OK;
    if (info.field == 0) return batch_launch_field<F31>(info, ws, blks, status, prof, s);
    return batch_launch_field<F64>(info, ws, blks, status, prof, s);
}

int ntt_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
               const uint64_t *key, uint64_t *out, cudaStream_t s) {
    (void)hdr;
    if (cfg.path == PA_PATH_NTT31) return launch_field<F31>(cfg, ws, prof, seed, key, out, s, 0);
    return launch_field<F64>(cfg, ws, prof, seed, key, out, s, 1);
}

}  // namespace pa
