// Measured issue-rate peaks for the roofline denominators of the integer paths.
//
// The NTT and direct kernels are bound by integer arithmetic, not by HBM, so their
// roofline is the rate at which this GPU executes the very operations they are built
// from. Each probe runs one of those operations, in registers, on independent chains in
// every thread of every SM (no memory traffic, no barriers, occupancy as the real kernel),
// and is timed with CUDA events:
//   PA_PEAK_NTT_BUTTERFLY  the 29-bit field's lazy Gentleman-Sande butterfly (F29::dif_bfly,
//                          the butterfly of every forward round of the NTT path);
//   PA_PEAK_NTT_MULADD     acc += x * y in the 29-bit field (a Montgomery product and a lazy
//                          addition: the pointwise products and transform-domain sums);
//   PA_PEAK_SHIFT_AND      acc ^= xw & funnel_shift(lo, hi, k) (the direct kernel's step);
//   PA_PEAK_MMA_S8         mma.sync m16n8k32 s8 x s8 -> s32 (the INT8 block path's MMA);
//   PA_PEAK_MMA_B1         mma.sync m16n8k256 b1 AND + POPC -> s32 (the binary form of the
//                          block contraction: one bit product per AND, summed by POPC);
//   PA_PEAK_NTT_GROUP28/29 radix-16 groups of the 28- or 29-bit field exactly as the NTT
//                          kernel's rounds run them (dif_group / dit_group of dft.cuh: the
//                          lazy reduction schedule, twiddles read from a shared-memory stage
//                          table), a forward and an inverse chain per thread.
// Each result is operations per second, one operation being one butterfly, one
// multiply-add, one shift-and-accumulate, or one multiply-accumulate of the MMA (an s8
// product, or a 1-bit AND product).
#include <stdint.h>

#include "common.cuh"
#include "dft.cuh"
#include "ntt_field.cuh"

namespace pa {
namespace {

constexpr int kProbeThreads = 512;
constexpr int kChains = 8;

// 2 kChains butterflies per iteration and thread.
__global__ void __launch_bounds__(kProbeThreads, 2) probe_butterfly(uint32_t *sink, uint32_t iters,
                                                                     F29::Tw w, uint32_t seed) {
    uint32_t a[kChains], b[kChains];
    const uint32_t x = seed ^ ((blockIdx.x * kProbeThreads + threadIdx.x) * 0x9E3779B9u);
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        a[c] = (x + 977u * c) & 0x0FFFFFFFu;         // < 2^28 < 4p
        b[c] = (x * 7u + 131u * c) & 0x0FFFFFFFu;
    }
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) F29::dif_bfly(a[c], b[c], w);
#pragma unroll
        for (int c = 0; c < kChains; ++c) F29::dif_bfly(b[c], a[c], w);
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r ^= a[c] ^ b[c];
    if (r == 0x9E3779B9u) sink[0] = r;  // keeps the chains live
}

// 32 butterflies per iteration and thread: iters radix-16 forward groups, then iters
// inverse groups, chained on the same 16 registers (a forward group's outputs meet both
// groups' input bounds, an inverse group's its own), with the twiddles of the stride-16
// round of a 256-point transform (j = lane mod 16).
template <class F>
__global__ void __launch_bounds__(kProbeThreads, 2) probe_group(uint32_t *sink, uint32_t iters,
                                                                 const typename F::Tw *__restrict__ tab,
                                                                 uint32_t seed) {
    using Tw = typename F::Tw;
    __shared__ Tw st[2][256];
    for (int i = threadIdx.x; i < 2 * 255; i += blockDim.x) st[i / 255][i % 255] = tab[i];
    __syncthreads();
    uint32_t x[16];
    const uint32_t v = seed ^ ((blockIdx.x * kProbeThreads + threadIdx.x) * 0x9E3779B9u);
#pragma unroll
    for (int k = 0; k < 16; ++k) x[k] = (v + 977u * k) % (4u * F::P);
    const int j = threadIdx.x & 15;
    for (uint32_t i = 0; i < iters; ++i) dif_group<F, 4>(x, st[0], j, 16);
    for (uint32_t i = 0; i < iters; ++i) dit_group<F, 4>(x, st[1], j, 16);
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) r ^= x[k];
    if (r == 0x9E3779B9u) sink[0] = r;
}

// 2 kChains multiply-adds per iteration and thread.
__global__ void __launch_bounds__(kProbeThreads, 2) probe_muladd(uint32_t *sink, uint32_t iters,
                                                                  uint32_t seed) {
    uint32_t acc[kChains], xv[kChains], yv[kChains];
    const uint32_t x = seed ^ ((blockIdx.x * kProbeThreads + threadIdx.x) * 0x9E3779B9u);
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
        acc[c] = 0;
        xv[c] = (x + 977u * c) & 0x0FFFFFFFu;
        yv[c] = (x * 7u + 131u * c) & 0x0FFFFFFFu;
    }
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) acc[c] = F29::add(acc[c], F29::mont(xv[c], yv[c]));
#pragma unroll
        for (int c = 0; c < kChains; ++c) xv[c] = F29::add(xv[c], F29::mont(acc[c], yv[c]));
    }
    uint32_t r = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) r ^= acc[c] ^ xv[c];
    if (r == 0x9E3779B9u) sink[0] = r;
}

// 32 shift-and-accumulate steps per iteration and thread (one 32 x 32 bit block of the
// direct kernel: 32 funnel shifts and 32 AND-XORs).
__global__ void __launch_bounds__(kProbeThreads, 2) probe_shift_and(uint32_t *sink, uint32_t iters,
                                                                     uint32_t seed) {
    uint32_t acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0;
    uint32_t lo = seed ^ ((blockIdx.x * kProbeThreads + threadIdx.x) * 0x9E3779B9u);
    uint32_t hi = lo * 0x85EBCA6Bu, xw = hi ^ 0x5BD1E995u;
    for (uint32_t i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] ^= xw & __funnelshift_r(lo, hi, k);
        const uint32_t t = lo;
        lo = hi;
        hi = xw;
        xw = t + i;
    }
    uint32_t r = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) r ^= acc[k];
    if (r == 0x9E3779B9u) sink[0] = r;
}

// kMma independent accumulator chains per warp; MMA operands stay in registers (changing
// each iteration so nothing is hoisted).
constexpr int kMma = 4;

__global__ void __launch_bounds__(kProbeThreads, 2) probe_mma_s8(uint32_t *sink, uint32_t iters,
                                                                  uint32_t seed) {
    uint32_t a[4], b[2];
    int32_t d[kMma][4];
    const uint32_t x = seed ^ ((blockIdx.x * kProbeThreads + threadIdx.x) * 0x9E3779B9u);
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = (x >> i) & 0x01010101u;
    b[0] = (x >> 5) & 0x01010101u;
    b[1] = (x >> 7) & 0x01010101u;
#pragma unroll
    for (int c = 0; c < kMma; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) d[c][i] = 0;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kMma; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
                "{%8,%9}, {%0,%1,%2,%3};"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
        const uint32_t t = a[0];  // rotate the A fragment (fixed indices: stays in registers)
        a[0] = a[1];
        a[1] = a[2];
        a[2] = a[3];
        a[3] = t ^ 0x01000000u;
    }
    int32_t r = 0;
#pragma unroll
    for (int c = 0; c < kMma; ++c) r ^= d[c][0] ^ d[c][1] ^ d[c][2] ^ d[c][3];
    if (r == 0x7654321) sink[0] = static_cast<uint32_t>(r);
}

__global__ void __launch_bounds__(kProbeThreads, 2) probe_mma_b1(uint32_t *sink, uint32_t iters,
                                                                  uint32_t seed) {
    uint32_t a[4], b[2];
    int32_t d[kMma][4];
    const uint32_t x = seed ^ ((blockIdx.x * kProbeThreads + threadIdx.x) * 0x9E3779B9u);
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = x * (2u * i + 1u);
    b[0] = x ^ 0x5BD1E995u;
    b[1] = x * 0x85EBCA6Bu;
#pragma unroll
    for (int c = 0; c < kMma; ++c)
#pragma unroll
        for (int i = 0; i < 4; ++i) d[c][i] = 0;
    for (uint32_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kMma; ++c)
            asm volatile(
                "mma.sync.aligned.m16n8k256.row.col.s32.b1.b1.s32.and.popc {%0,%1,%2,%3}, "
                "{%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
                : "+r"(d[c][0]), "+r"(d[c][1]), "+r"(d[c][2]), "+r"(d[c][3])
                : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
        const uint32_t t = a[0];
        a[0] = a[1];
        a[1] = a[2];
        a[2] = a[3];
        a[3] = t + 0x9E3779B9u;
    }
    int32_t r = 0;
#pragma unroll
    for (int c = 0; c < kMma; ++c) r ^= d[c][0] ^ d[c][1] ^ d[c][2] ^ d[c][3];
    if (r == 0x7654321) sink[0] = static_cast<uint32_t>(r);
}

// Twiddles for the group probe: canonical residues (powers of the field's 16th root of
// unity) with their Shoup quotients, 255 per direction. The cost of a group does not depend
// on the values, only on the reads and the arithmetic.
template <class F>
void group_tables(typename F::Tw *out) {
    const uint64_t p = F::P;
    uint64_t w = 1;
    for (int i = 0; i < 2 * 255; ++i) {
        out[i].w = static_cast<uint32_t>(w);
        out[i].q = static_cast<uint32_t>((w << 32) / p);
        w = w * F::kRoot16 % p;
    }
}

// Launches probe `which` with `iters` iterations per thread; returns operations per launch.
double probe_launch(int which, uint32_t iters, unsigned grid, uint32_t *sink, const void *tabs,
                    cudaStream_t s) {
    const double threads = double(grid) * kProbeThreads;
    if (which == PA_PEAK_NTT_GROUP28) {
        probe_group<F28><<<grid, kProbeThreads, 0, s>>>(sink, iters, static_cast<const F28::Tw *>(tabs),
                                                        0x1234567u);
        return threads * iters * 64.0;
    }
    if (which == PA_PEAK_NTT_GROUP29) {
        probe_group<F29><<<grid, kProbeThreads, 0, s>>>(sink, iters, static_cast<const F29::Tw *>(tabs),
                                                        0x1234567u);
        return threads * iters * 64.0;
    }
    if (which == PA_PEAK_NTT_BUTTERFLY) {
        F29::Tw w;
        w.w = 123456789u;  // a canonical residue with its Shoup quotient
        w.q = static_cast<uint32_t>((uint64_t(w.w) << 32) / F29::P);
        probe_butterfly<<<grid, kProbeThreads, 0, s>>>(sink, iters, w, 0x1234567u);
        return threads * iters * 2.0 * kChains;
    }
    if (which == PA_PEAK_NTT_MULADD) {
        probe_muladd<<<grid, kProbeThreads, 0, s>>>(sink, iters, 0x1234567u);
        return threads * iters * 2.0 * kChains;
    }
    if (which == PA_PEAK_MMA_S8) {
        probe_mma_s8<<<grid, kProbeThreads, 0, s>>>(sink, iters, 0x1234567u);
        return threads / 32.0 * iters * kMma * (16.0 * 8.0 * 32.0);
    }
    if (which == PA_PEAK_MMA_B1) {
        probe_mma_b1<<<grid, kProbeThreads, 0, s>>>(sink, iters, 0x1234567u);
        return threads / 32.0 * iters * kMma * (16.0 * 8.0 * 256.0);
    }
    probe_shift_and<<<grid, kProbeThreads, 0, s>>>(sink, iters, 0x1234567u);
    return threads * iters * 32.0;
}

}  // namespace
}  // namespace pa

extern "C" int pa_probe_peak(int which, double *ops_per_s, double *ms) {
    using namespace pa;
    if (!ops_per_s || which < PA_PEAK_NTT_BUTTERFLY || which > PA_PEAK_NTT_GROUP29) return PA_ERR_INVALID;
    int dev = 0, sms = 0, per_sm = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    PA_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const void *fn = which == PA_PEAK_NTT_BUTTERFLY ? reinterpret_cast<const void *>(probe_butterfly)
                     : which == PA_PEAK_NTT_MULADD  ? reinterpret_cast<const void *>(probe_muladd)
                     : which == PA_PEAK_MMA_S8      ? reinterpret_cast<const void *>(probe_mma_s8)
                     : which == PA_PEAK_MMA_B1      ? reinterpret_cast<const void *>(probe_mma_b1)
                     : which == PA_PEAK_NTT_GROUP28 ? reinterpret_cast<const void *>(probe_group<F28>)
                     : which == PA_PEAK_NTT_GROUP29 ? reinterpret_cast<const void *>(probe_group<F29>)
                                                    : reinterpret_cast<const void *>(probe_shift_and);
    PA_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kProbeThreads, 0));
    const unsigned grid = static_cast<unsigned>((per_sm > 0 ? per_sm : 1) * sms);
    uint32_t *sink = nullptr;
    void *tabs = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t e = cudaMalloc(&sink, 256);
    if (e == cudaSuccess && (which == PA_PEAK_NTT_GROUP28 || which == PA_PEAK_NTT_GROUP29)) {
        F31::Tw host[2 * 255];  // the 32-bit fields share this twiddle layout
        if (which == PA_PEAK_NTT_GROUP28)
            group_tables<F28>(host);
        else
            group_tables<F29>(host);
        e = cudaMalloc(&tabs, sizeof(host));
        if (e == cudaSuccess) e = cudaMemcpy(tabs, host, sizeof(host), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&a);
    if (e == cudaSuccess) e = cudaEventCreate(&b);
    double best = 0.0, best_ms = 0.0;
    if (e == cudaSuccess) {
        // size the launch to about 20 ms from a short one, then take the fastest of three
        uint32_t iters = 256;
        float t = 0.f;
        for (int r = 0; r < 2 && e == cudaSuccess; ++r) {  // warm-up and sizing
            cudaEventRecord(a, s);
            probe_launch(which, iters, grid, sink, tabs, s);
            cudaEventRecord(b, s);
            e = cudaEventSynchronize(b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
        }
        if (e == cudaSuccess && t > 0.f) {
            double scaled = double(iters) * 20.0 / double(t);
            iters = static_cast<uint32_t>(scaled < 256.0 ? 256.0 : (scaled > 4.0e6 ? 4.0e6 : scaled));
        }
        for (int r = 0; r < 3 && e == cudaSuccess; ++r) {
            cudaEventRecord(a, s);
            const double ops = probe_launch(which, iters, grid, sink, tabs, s);
            cudaEventRecord(b, s);
            e = cudaEventSynchronize(b);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
            if (e == cudaSuccess && t > 0.f && ops / (t * 1e-3) > best) {
                best = ops / (t * 1e-3);
                best_ms = t;
            }
        }
        if (e == cudaSuccess) e = cudaGetLastError();
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    if (s) cudaStreamDestroy(s);
    cudaFree(sink);
    cudaFree(tabs);
    if (e != cudaSuccess) return cuda_fail(e);
    *ops_per_s = best;
    if (ms) *ms = best_ms;
    return PA_OK;
}
