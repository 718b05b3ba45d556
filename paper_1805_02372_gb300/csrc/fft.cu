// Floating-point transform path: the paper's FFT route (Sec. 3, Steps 1-3) on
// sub-blocks short enough that a proven rounding-error bound stays below 1/2, so
// rounding recovers every integer coefficient exactly (Sec. 3 replaces the paper's
// empirical FP32 length limit with a proof). FP64 butterflies are used only for tile
// geometries whose FP32 bound is not below 1/2.
//
// One CTA per tile (key tile a of length L, seed window w of length L+M, transform
// size N <= 2^12): complex FFTs of a and w (radix-2 stages, two per shared-memory
// round trip), the pointwise product, the inverse FFT, then for each wanted
// coefficient v = Re(c_k)/N: rint(v), its low bit XORed into the output, and
// |v - rint(v)| folded into the plan's worst-residual word.
//
// Bound (unnormalised DFT F, computed with radix-2 butterflies and twiddles of error
// <= mu; Higham, Accuracy and Stability of Numerical Algorithms, 2nd ed., Thm 24.2:
// ||fl(Fz) - Fz||_2 <= alpha ||Fz||_2, alpha = k eta / (1 - k eta), k = log2 N,
// eta = mu + gamma_4 (sqrt2 + mu); complex products off by <= sqrt2 gamma_2):
//   |c^_k - c_k| <= ||a||_2 ||w||_2 (2 alpha + alpha^2 + sqrt2 gamma_2 (1+alpha)^2)
//                 + alpha (1 + sqrt2 gamma_2)(1 + alpha)(||a||_1 + alpha sqrt(N) ||a||_2) ||w||_2,
// the first line from the forward transforms and the product (||u (.) v||_1 <=
// ||u||_2 ||v||_2, |(F^* v)_k| <= ||v||_1), the second from the inverse transform
// (||F^* e||_inf <= ||e||_2 ... with ||X^||_inf <= ||a||_1 + ||e_a||_2). For 0/1 data
// the worst case is every bit set: ||a||_1 = L, ||a||_2 = sqrt(L), ||w||_2 = sqrt(L+M).
#include <math.h>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "dft.cuh"
#include "tiles.cuh"

namespace pa {

constexpr int kFftLogMax = 12;  // tiles live in one CTA's shared memory
constexpr int kFftThreads = 512;

template <class R>
struct Vec2;
template <>
struct Vec2<float> {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <class R>
struct CRing {
    using T = typename Vec2<R>::type;
    using Tw = T;
    __device__ static __forceinline__ T add(T a, T b) {
        T r;
        r.x = a.x + b.x;
        r.y = a.y + b.y;
        return r;
    }
    __device__ static __forceinline__ T sub(T a, T b) {
        T r;
        r.x = a.x - b.x;
        r.y = a.y - b.y;
        return r;
    }
    __device__ static __forceinline__ T mul_tw(T a, Tw w) {
        T r;
        r.x = a.x * w.x - a.y * w.y;
        r.y = a.x * w.y + a.y * w.x;
        return r;
    }
    __device__ static __forceinline__ void dif_bfly(T &a, T &b, Tw w) {
        const T s = add(a, b);
        b = mul_tw(sub(a, b), w);
        a = s;
    }
    __device__ static __forceinline__ void dit_bfly(T &a, T &b, Tw w) {
        const T t = mul_tw(b, w);
        b = sub(a, t);
        a = add(a, t);
    }
};

// ---------------------------------------------------------------- the bound

double fft_rounding_bound(uint32_t logn, uint64_t L, uint64_t M, bool fp64) {
    const double u = fp64 ? ldexp(1.0, -53) : ldexp(1.0, -24);
    // twiddles: cos/sin evaluated in double (error <= 1 ulp of double) and, for FP32,
    // rounded once to float
    const double mu = fp64 ? 2.0 * u : u * (1.0 + ldexp(1.0, -20));
    auto gamma = [u](double k) { return k * u / (1.0 - k * u); };
    const double eta = mu + gamma(4) * (sqrt(2.0) + mu);
    const double k = static_cast<double>(logn);
    if (k * eta >= 1.0) return INFINITY;
    const double alpha = k * eta / (1.0 - k * eta);
    const double g2 = sqrt(2.0) * gamma(2);
    const double N = ldexp(1.0, static_cast<int>(logn));
    const double a1 = static_cast<double>(L), a2 = sqrt(static_cast<double>(L));
    const double w2 = sqrt(static_cast<double>(L + M));
    const double t1 = a2 * w2 * (2 * alpha + alpha * alpha + g2 * (1 + alpha) * (1 + alpha));
    const double t2 = alpha * (1 + g2) * (1 + alpha) * (a1 + alpha * sqrt(N) * a2) * w2;
    return t1 + t2;
}

namespace {

// ---------------------------------------------------------------- twiddle tables

struct FftTables {
    void *f32 = nullptr, *f64 = nullptr;
};
std::mutex g_fft_mu;
FftTables g_fft[64];

int fft_tables(int fp64, const void **out) {
    int dev = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_fft_mu);
    FftTables &t = g_fft[dev];
    void *&slot = fp64 ? t.f64 : t.f32;
    if (!slot) {
        const size_t half = size_t(1) << (kFftLogMax - 1);
        const double Nmax = ldexp(1.0, kFftLogMax);
        const double twopi = 6.283185307179586476925286766559;
        std::vector<double2> d(half);
        std::vector<float2> f(half);
        for (size_t j = 0; j < half; ++j) {
            // w^j = exp(-2 pi i j / Nmax)
            const double th = twopi * static_cast<double>(j) / Nmax;
            d[j].x = cos(th);
            d[j].y = -sin(th);
            f[j].x = static_cast<float>(d[j].x);
            f[j].y = static_cast<float>(d[j].y);
        }
        const size_t bytes = half * (fp64 ? sizeof(double2) : sizeof(float2));
        void *p = nullptr;
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e == cudaSuccess)
            e = cudaMemcpy(p, fp64 ? static_cast<const void *>(d.data()) : f.data(), bytes,
                           cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            cudaFree(p);
            return cuda_fail(e);
        }
        slot = p;
    }
    *out = slot;
    return PA_OK;
}

// Tile (I, J) from the flat tile index: pairs are ordered output-tile major.
struct FftGrid {
    uint64_t n, m, L, M, tiles_in;
};

__device__ __forceinline__ TilePair tile_at(const FftGrid &g, uint64_t idx) {
    const uint64_t I = idx / g.tiles_in, J = idx - I * g.tiles_in;
    TilePair p;
    const uint64_t i0 = I * g.M, j0 = J * g.L;
    p.key_bit0 = static_cast<int64_t>(j0);
    p.key_len = (g.n - j0 < g.L) ? g.n - j0 : g.L;
    p.K0 = static_cast<uint32_t>(g.L);
    p.win_bit0 = static_cast<int64_t>(g.n) - 1 + static_cast<int64_t>(i0) - static_cast<int64_t>(j0) -
                 static_cast<int64_t>(g.L);
    p.win_len = g.L + g.M;
    p.out_bit0 = i0;
    p.out_len = static_cast<uint32_t>((g.m - i0 < g.M) ? g.m - i0 : g.M);
    p.blk = 0;
    p.pad = 0;
    return p;
}

__device__ __forceinline__ float rint_(float v) { return rintf(v); }
__device__ __forceinline__ double rint_(double v) { return rint(v); }

template <class R>
__global__ void __launch_bounds__(kFftThreads) fft_tile(FftGrid g, uint64_t tile0, BlockPtrs bp,
                                                        int logN,
                                                        const typename CRing<R>::Tw *__restrict__ tab,
                                                        unsigned long long *residual_bits) {
    using F = CRing<R>;
    using T = typename F::T;
    extern __shared__ __align__(16) unsigned char smraw[];
    __shared__ R red[kFftThreads / 32];
    const int N = 1 << logN;
    T *st = reinterpret_cast<T *>(smraw);
    T *sm = st + N;  // column 0: key tile, column 1: window
    const ColMajor lay{ColMajor::stride(N)};
    const TilePair pr = tile_at(g, tile0 + blockIdx.x);
    load_stage_tables<F>(st, tab, logN, kFftLogMax);
    for (int t = threadIdx.x; t < N; t += blockDim.x) {
        T a, w;
        a.x = static_cast<R>(key_bit(pr, bp, t));
        a.y = 0;
        w.x = static_cast<R>(win_bit(pr, bp, t));
        w.y = 0;
        sm[lay.at(t, 0)] = a;
        sm[lay.at(t, 1)] = w;
    }
    __syncthreads();
    dif_columns<F, false>(sm, lay, logN, 1, st);
    for (int t = threadIdx.x; t < N; t += blockDim.x)
        sm[lay.at(t, 1)] = F::mul_tw(sm[lay.at(t, 0)], sm[lay.at(t, 1)]);
    __syncthreads();
    for (int t = threadIdx.x; t < N - 1; t += blockDim.x) st[t].y = -st[t].y;  // conjugate twiddles
    __syncthreads();
    dit_columns<F, false>(sm + lay.cs, lay, logN, 0, st);
    const R inv_n = static_cast<R>(1) / static_cast<R>(N);  // power of two: exact
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t nw = (pr.out_len + 31) / 32;
    R worst = 0;
    for (uint32_t wv = warp; wv < nw; wv += blockDim.x / 32) {
        const uint32_t v = wv * 32 + lane;
        uint32_t bit = 0;
        if (v < pr.out_len) {
            const R val = sm[lay.at(pr.K0 + v, 1)].x * inv_n;
            const R r = rint_(val);
            worst = fmax(worst, fabs(val - r));
            bit = static_cast<uint32_t>(static_cast<long long>(r)) & 1u;
        }
        const uint32_t word = __ballot_sync(0xFFFFFFFFu, bit);
        if (lane == 0 && word) atomicXor(bp.out32 + (pr.out_bit0 >> 5) + wv, word);
    }
    for (int o = 16; o; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xFFFFFFFFu, worst, o));
    if (lane == 0) red[warp] = worst;
    __syncthreads();
    if (threadIdx.x == 0) {
        R m = 0;
        for (int i = 0; i < static_cast<int>(blockDim.x / 32); ++i) m = fmax(m, red[i]);
        const double md = static_cast<double>(m);
        atomicMax(residual_bits, static_cast<unsigned long long>(__double_as_longlong(md)));
    }
}

bool fft_ok(uint32_t logn, uint64_t L, uint64_t M, bool fp64) {
    return fft_rounding_bound(logn, L, M, fp64) < 0.5;
}

}  // namespace

// Largest proven FP32 key tile for transform size 2^logn and output tile M.
static uint64_t max_L32(uint32_t logn, uint64_t M) {
    const uint64_t N = uint64_t(1) << logn;
    if (M + 32 > N) return 0;
    uint64_t L = ((N - M) / 32) * 32;
    while (L >= 32 && !fft_ok(logn, L, M, false)) L -= 32;
    return L >= 32 ? L : 0;
}

int fft_plan(uint64_t n, uint64_t m, const pa_opts *o, TransformCfg *c) {
    *c = TransformCfg();
    const uint32_t force = o ? o->log2_transform : 0;
    const uint64_t Mf = o ? o->tile_out : 0, Lf = o ? o->tile_in : 0;
    const bool want64 = o && o->force_fp64;
    if (force > kFftLogMax) return PA_ERR_UNSUPPORTED;
    if (force && (Lf || Mf)) {
        // Caller-chosen geometry: FP32 when proven, FP64 where the FP32 bound fails.
        const uint64_t N = uint64_t(1) << force;
        const uint64_t M = Mf ? round_up(Mf, 64) : 64, L = Lf ? round_up(Lf, 32) : 32;
        if (L + M > N) return PA_ERR_INVALID;
        bool fp64 = want64 || !fft_ok(force, L, M, false);
        if (fp64 && !fft_ok(force, L, M, true)) return PA_ERR_PRECISION;
        c->log2n = force;
        c->L = L;
        c->M = M;
        c->fp64 = fp64;
    } else {
        double best = 1e300;
        const uint64_t mcap = round_up(m, 64), ncap = round_up(n, 32);
        for (uint32_t k = 6; k <= kFftLogMax; ++k) {
            if (force && k != force) continue;
            const uint64_t N = uint64_t(1) << k;
            for (uint64_t M = 64; M + 32 <= N; M += 64) {
                if (M > mcap) break;
                uint64_t L = max_L32(k, M);
                if (want64) L = ((N - M) / 32) * 32;
                if (!L) continue;
                if (L > ncap) L = ncap;
                const double pairs = double(ceil_div(n, L)) * double(ceil_div(m, M));
                const double cost = pairs * double(N) * (k + 2) * (want64 ? 40.0 : 1.0);
                if (cost < best) {
                    best = cost;
                    c->log2n = k;
                    c->L = L;
                    c->M = M;
                }
            }
        }
        if (best >= 1e300) return PA_ERR_UNSUPPORTED;
        c->fp64 = want64;
    }
    c->tiles_in = ceil_div(n, c->L);
    c->tiles_out = ceil_div(m, c->M);
    c->bound = fft_rounding_bound(c->log2n, c->L, c->M, c->fp64);
    c->passes = 1;
    c->radix_log2[0] = c->log2n;
    return PA_OK;
}

size_t fft_workspace(const TransformCfg &) { return 0; }

int fft_prepare(int fp64) {
    const void *t = nullptr;
    return fft_tables(fp64, &t);
}

int fft_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
               const uint64_t *key, uint64_t *out, cudaStream_t s) {
    (void)ws;
    const TransformCfg &c = cfg.tr;
    const void *tab = nullptr;
    int rc = fft_tables(c.fp64, &tab);
    if (rc != PA_OK) return rc;
    BlockPtrs bp{reinterpret_cast<const uint32_t *>(key), reinterpret_cast<const uint32_t *>(seed),
                 reinterpret_cast<uint32_t *>(out), cfg.n, cfg.m};
    FftGrid g{cfg.n, cfg.m, c.L, c.M, c.tiles_in};
    const int logN = static_cast<int>(c.log2n);
    const uint64_t tiles = c.tiles_in * c.tiles_out;
    prof_begin(prof, K_MEMSET, s);
    PA_CUDA_TRY(cudaMemsetAsync(out, 0, ceil_div(cfg.m, 64) * 8, s));
    prof_end(prof, s);
    const uint64_t chunk = 1u << 30;
    if (c.fp64) {
        const size_t smem = ((size_t(1) << logN) + ColMajor::words(1 << logN, 2)) * sizeof(double2);
        PA_CUDA_TRY(cudaFuncSetAttribute(fft_tile<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
        for (uint64_t t0 = 0; t0 < tiles; t0 += chunk) {
            const uint64_t cnt = tiles - t0 < chunk ? tiles - t0 : chunk;
            prof_begin(prof, K_FFT_TILE, s);
            fft_tile<double><<<static_cast<unsigned>(cnt), kFftThreads, smem, s>>>(
                g, t0, bp, logN, static_cast<const double2 *>(tab), &hdr->residual_bits);
            prof_end(prof, s);
        }
    } else {
        const size_t smem = ((size_t(1) << logN) + ColMajor::words(1 << logN, 2)) * sizeof(float2);
        PA_CUDA_TRY(cudaFuncSetAttribute(fft_tile<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
        for (uint64_t t0 = 0; t0 < tiles; t0 += chunk) {
            const uint64_t cnt = tiles - t0 < chunk ? tiles - t0 : chunk;
            prof_begin(prof, K_FFT_TILE, s);
            fft_tile<float><<<static_cast<unsigned>(cnt), kFftThreads, smem, s>>>(
                g, t0, bp, logN, static_cast<const float2 *>(tab), &hdr->residual_bits);
            prof_end(prof, s);
        }
    }
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace pa

extern "C" int pa_fft_rounding_bound(uint32_t log2_transform, uint64_t tile_in, uint64_t tile_out,
                                     int fp64, double *bound) {
    if (!bound || log2_transform == 0 || log2_transform > 40) return PA_ERR_INVALID;
    *bound = pa::fft_rounding_bound(log2_transform, tile_in, tile_out, fp64 != 0);
    return PA_OK;
}
