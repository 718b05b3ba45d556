// Direct path: the Toeplitz hash as a bit-packed GF(2) matrix-vector product
// (Sec. 2.1 Eq. 1: T[i][j] = s[n-1+i-j], y = T x mod 2).
//
// Reversing the key, xr[j] = x[n-1-j], turns row i of T into the seed window that
// starts at bit i:  y[i] = parity( sum_j xr[j] AND s[i+j] ).  A thread owns 32
// consecutive rows (one 32-bit output word) and a chunk of 32-bit key words; for
// key word q the 32 row windows are funnel shifts of two adjacent seed words, so
// each 32x32 bit block costs 32 SHF + 32 LOP3 (acc ^= xw & window). The parity of
// each row's accumulator (one POPC) is packed back into an output word; partial
// words from different key chunks are merged with atomicXor (the XOR merge of
// Eq. finalkey). Key chunks and seed windows are staged in shared memory by the
// TMA engine (cp.async.bulk + mbarrier).
#include <mutex>

#include "common.cuh"

namespace pa {
namespace {

constexpr int kThreads = 128;      // 4 warps; one row group (32 rows) per thread
constexpr int kRowGroups = kThreads;

// xr[q] bit c = x[n-1-32q-c] (0 where that index is negative); zero padding past
// ceil(n/32) words. The same launch zeroes zero_words 64-bit words at `zero` (the output of
// a kernel that merges its partial results with atomicXor), one operation fewer per hash.
__global__ void reverse_key_kernel(const uint32_t *__restrict__ key32, uint64_t key_buf_words32,
                                   uint64_t n, uint32_t *__restrict__ xr, uint64_t words,
                                   uint64_t words_pad, uint64_t *__restrict__ zero, uint64_t zero_words) {
    const uint64_t span = words_pad > zero_words ? words_pad : zero_words;
    for (uint64_t q = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; q < span;
         q += uint64_t(gridDim.x) * blockDim.x) {
        if (q < zero_words) zero[q] = 0;
        if (q >= words_pad) continue;
        uint32_t v = 0;
        if (q < words) {
            int64_t lo = static_cast<int64_t>(n) - 1 - 32 * static_cast<int64_t>(q) - 31;
            v = __brev(bits32_at(key32, key_buf_words32, lo));
        }
        xr[q] = v;
    }
}

__global__ void __launch_bounds__(kThreads) direct_kernel(
    const uint32_t *__restrict__ seed32, uint64_t seed_words32, const uint32_t *__restrict__ xr,
    uint32_t kc, uint64_t m, uint32_t *__restrict__ out32, uint64_t out_words32, int use_atomic,
    int *status) {
    extern __shared__ __align__(128) uint32_t sm[];
    __shared__ __align__(8) uint64_t bar;
    uint32_t *skey = sm;
    uint32_t *sseed = sm + kc;

    const uint64_t g0 = uint64_t(blockIdx.x) * kRowGroups;  // first row group (= seed word)
    const uint64_t k0 = uint64_t(blockIdx.y) * kc;          // first key word
    const uint64_t sb = g0 + k0;                            // first seed word needed
    const uint32_t count = kRowGroups + kc + 4;             // seed words staged
    const uint64_t avail = seed_words32 > sb ? seed_words32 - sb : 0;
    const uint32_t bulk = static_cast<uint32_t>(avail < count ? avail : count) & ~3u;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (kc + bulk) * 4u);
        bulk_g2s(skey, xr + k0, kc * 4u, &bar);
        if (bulk) bulk_g2s(sseed, seed32 + sb, bulk * 4u, &bar);
    }
    for (uint32_t t = bulk + threadIdx.x; t < count; t += kThreads)
        sseed[t] = (sb + t < seed_words32) ? __ldg(seed32 + sb + t) : 0u;
    const bool ok = mbar_wait_bounded(&bar, 0, status);
    __syncthreads();
    if (!ok) return;

    uint32_t acc[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) acc[k] = 0;

    const uint32_t *sp = sseed + threadIdx.x;
    uint32_t lo = sp[0];
#pragma unroll 2
    for (uint32_t q = 0; q < kc; ++q) {
        const uint32_t xw = skey[q];
        const uint32_t hi = sp[q + 1];
#pragma unroll
        for (int k = 0; k < 32; ++k) acc[k] ^= xw & __funnelshift_r(lo, hi, k);
        lo = hi;
    }

    uint32_t res = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) res |= (__popc(acc[k]) & 1u) << k;

    const uint64_t g = g0 + threadIdx.x;
    if (g < out_words32) {
        const uint64_t row0 = g * 32;
        if (row0 + 32 > m) res = (m > row0) ? (res & ((1u << (m - row0)) - 1u)) : 0u;
        if (use_atomic)
            atomicXor(out32 + g, res);
        else
            out32[g] = res;
    }
}

}  // namespace

int direct_plan(uint64_t n, uint64_t m, DirectCfg *c) {
    c->key_words32 = ceil_div(n, 32);
    const uint64_t out_words32 = 2 * ceil_div(m, 64);
    const uint64_t gx = ceil_div(out_words32, kRowGroups);
    const uint64_t target = uint64_t(kNumSMsGB300) * 8 * 4;  // ~4 waves of 8 CTAs per SM
    uint64_t kc = ceil_div(c->key_words32 * gx, target);
    kc = round_up(kc < 32 ? 32 : kc, 4);
    if (kc > 4096) kc = 4096;
    const uint64_t kw4 = round_up(c->key_words32, 4);
    if (kc > kw4) kc = kw4;
    const uint64_t gy = ceil_div(c->key_words32, kc);
    if (gx > 0x7fffffffull || gy > 65535) return PA_ERR_UNSUPPORTED;
    c->kc = static_cast<uint32_t>(kc);
    c->grid_x = static_cast<uint32_t>(gx);
    c->grid_y = static_cast<uint32_t>(gy);
    c->key_words32_pad = gy * kc;
    return PA_OK;
}

void reverse_key_launch(const uint64_t *key, uint64_t n, uint32_t *xr, uint64_t words,
                        uint64_t words_pad, cudaStream_t s, uint64_t *zero, uint64_t zero_words) {
    uint64_t blocks = ceil_div(words_pad > zero_words ? words_pad : zero_words, 256);
    if (blocks > 4096) blocks = 4096;
    if (blocks == 0) blocks = 1;
    reverse_key_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(
        reinterpret_cast<const uint32_t *>(key), 2 * ceil_div(n, 64), n, xr, words, words_pad,
        zero, zero ? zero_words : 0);
}

size_t direct_workspace(const DirectCfg &c) { return round_up(c.key_words32_pad * 4, 256); }

int direct_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
                  const uint64_t *key, uint64_t *out, cudaStream_t s) {
    const DirectCfg &c = cfg.direct;
    const uint64_t n = cfg.n, m = cfg.m;
    uint32_t *xr = static_cast<uint32_t *>(ws);
    const uint64_t out_words64 = ceil_div(m, 64);
    const int use_atomic = c.grid_y > 1;
    // the key reversal also zeroes the output when the key chunks merge by atomicXor
    prof_begin(prof, K_REVERSE_KEY, s);
    reverse_key_launch(key, n, xr, c.key_words32, c.key_words32_pad, s, use_atomic ? out : nullptr,
                       out_words64);
    prof_end(prof, s);
    const size_t smem = (size_t(c.kc) + kRowGroups + c.kc + 4) * 4;
    if (smem > 48 * 1024)
        PA_CUDA_TRY(cudaFuncSetAttribute(direct_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
    dim3 grid(c.grid_x, c.grid_y);
    prof_begin(prof, K_DIRECT, s);
    direct_kernel<<<grid, kThreads, smem, s>>>(
        reinterpret_cast<const uint32_t *>(seed), 2 * ceil_div(n + m - 1, 64), xr, c.kc, m,
        reinterpret_cast<uint32_t *>(out), 2 * out_words64, use_atomic, &hdr->status);
    prof_end(prof, s);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace pa

// ---------------------------------------------------------------- no-allocation entry point
//
// Some callers cannot call cudaMalloc: a post-processing pipeline that reserved its device
// memory once at start-up and forbids allocation afterwards (allocation can synchronise the
// device and stall the real-time stream), a host process whose memory arena belongs to
// another framework, or code that must not fail on out-of-memory halfway through a key.
// For them, pa_hash_direct_static runs the direct kernel with its scratch (the reversed
// key and the status word) in the fixed array below, which every GPU that loads this
// library holds until the process exits. Inputs and outputs remain the caller's.
namespace pa {
namespace {

constexpr uint64_t kStaticMaxKeyBits = uint64_t(1) << 25;  // n <= 33,554,432 key bits
constexpr uint64_t kStaticHeaderWords = kHeaderBytes / 4;  // status word area
// reversed key of up to kStaticMaxKeyBits bits, padded to the largest key chunk (4096 words)
constexpr uint64_t kStaticScratchWords = kStaticHeaderWords + kStaticMaxKeyBits / 32 + 4096;

static __device__ __align__(256) uint32_t g_static_scratch[kStaticScratchWords];

std::mutex g_static_mu;
uint32_t *g_static_ptr[64] = {nullptr};

// Device address of the array on the current device. Outside stream capture it is looked
// up on every call (cheap, and never stale: a device reset or a new primary context gives
// the array a new address); during capture only the address cached by an earlier call on
// this device is used, and a first call under capture is refused.
int static_scratch(cudaStream_t s, uint32_t **out) {
    int dev = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return PA_ERR_INVALID;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    PA_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (cs != cudaStreamCaptureStatusNone) {
        if (!g_static_ptr[dev]) return PA_ERR_INVALID;
        *out = g_static_ptr[dev];
        return PA_OK;
    }
    uint32_t *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_static_scratch);
    if (e != cudaSuccess) {
        g_static_ptr[dev] = nullptr;
        return cuda_fail(e);
    }
    g_static_ptr[dev] = p;
    *out = p;
    return PA_OK;
}

}  // namespace
}  // namespace pa

extern "C" int pa_hash_direct_static(uint64_t n, uint64_t m, const uint64_t *seed_bits,
                                     const uint64_t *key_bits, uint64_t *out_bits, void *stream) {
    using namespace pa;
    if (n == 0 || m == 0 || !seed_bits || !key_bits || !out_bits) return PA_ERR_INVALID;
    if (((reinterpret_cast<uintptr_t>(seed_bits) | reinterpret_cast<uintptr_t>(key_bits) |
          reinterpret_cast<uintptr_t>(out_bits)) & 15u) != 0)
        return PA_ERR_ALIGN;
    if (n > kStaticMaxKeyBits || m > (uint64_t(1) << 40)) return PA_ERR_TOO_LARGE;
    PlanCfg cfg;
    cfg.n = n;
    cfg.m = m;
    cfg.path = PA_PATH_DIRECT;
    int rc = direct_plan(n, m, &cfg.direct);
    if (rc != PA_OK) return rc;
    if (kStaticHeaderWords + cfg.direct.key_words32_pad > kStaticScratchWords) return PA_ERR_TOO_LARGE;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *scratch = nullptr;
    rc = static_scratch(s, &scratch);
    if (rc != PA_OK) return rc;
    // the status word must start at zero; the reversed key is fully rewritten below
    PA_CUDA_TRY(cudaMemsetAsync(scratch, 0, sizeof(DevHeader), s));
    return direct_launch(cfg, scratch + kStaticHeaderWords, reinterpret_cast<DevHeader *>(scratch),
                         nullptr, seed_bits, key_bits, out_bits, s);
}

extern "C" int pa_direct_static_status(void *stream) {
    using namespace pa;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *scratch = nullptr;
    int rc = static_scratch(s, &scratch);
    if (rc != PA_OK) return rc;
    PA_CUDA_TRY(cudaStreamSynchronize(s));
    int status = 0;
    PA_CUDA_TRY(cudaMemcpy(&status, scratch, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
        const int zero = 0;
        PA_CUDA_TRY(cudaMemcpy(scratch, &zero, sizeof(int), cudaMemcpyHostToDevice));
    }
    return status;
}
