// Block-Toeplitz path: the hash as the one dense form of the computation,
// Y[:, I] = sum_d T_d X[:, I-d] with b x b Toeplitz tiles T_d[a][c] = s[n-1+b*d+a-c]
// (the row split of Eq. Ti/Eq. Tij taken down to tiles of b rows), on the tensor
// cores in INT8 with INT32 accumulation, then mod 2.
//
// As a GEMM: C[a][I] = sum_k A[a][k] B[k][I] with A[a][k] = s[n-1+a+k] (every b-wide
// slab of k is one T_d, columns reversed) and B[k][I] = x[b*I-k] = xr[n-1-b*I+k]
// (xr the reversed key). Both operands are expanded on the fly from bits: the four
// INT8 values of one fragment register are four consecutive bits of the seed or of
// the reversed key, spread to bytes with one multiply and one mask. Counts are at
// most n < 2^31, so INT32 accumulation is exact; y[b*I+a] = C[a][I] & 1.
//
// sm_103a has no tcgen05 INT8 MMA kind, so the contraction uses the warp-level
// mma.sync.m16n8k32.s32.s8.s8.s32. A CTA (4 warps) owns b rows x 8192/b output
// blocks (8192 outputs) and a chunk of the contraction; chunks are XOR-merged.
#include "common.cuh"

namespace pa {
namespace {

constexpr int kBlkThreads = 128;
constexpr int kTileOutputs = 8192;

__device__ __forceinline__ uint32_t nib(const uint32_t *w, int p) {
    return __funnelshift_r(w[p >> 5], w[(p >> 5) + 1], p & 31) & 0xFu;
}
// Four bits -> four bytes (bit i to byte i): shifted copies do not overlap, no carries.
__device__ __forceinline__ uint32_t spread(uint32_t v) { return (v * 0x00204081u) & 0x01010101u; }

__device__ __forceinline__ void mma_s8(int (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                       uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Stage `words` 32-bit words of a bit string starting at bit `base` (bits outside
// [0, valid) read as 0).
__device__ __forceinline__ void stage_bits(uint32_t *dst, int words, const uint32_t *__restrict__ src,
                                           uint64_t src_words, int64_t base, uint64_t valid) {
    for (int w = threadIdx.x; w < words; w += blockDim.x) {
        const int64_t p = base + 32 * static_cast<int64_t>(w);
        uint32_t v = bits32_at(src, src_words, p);
        // clear positions < 0 (bits32_at reads them as 0) and >= valid
        if (p + 32 > static_cast<int64_t>(valid)) {
            const int64_t keep = static_cast<int64_t>(valid) - p;
            v = keep <= 0 ? 0u : (keep >= 32 ? v : (v & ((1u << keep) - 1u)));
        }
        dst[w] = v;
    }
}

template <int B>
__global__ void __launch_bounds__(kBlkThreads) block_mma_kernel(
    const uint32_t *__restrict__ seed32, uint64_t seed_words32, const uint32_t *__restrict__ xr,
    uint64_t xr_words32, uint64_t n, uint64_t m, uint32_t kc, uint32_t *__restrict__ out32,
    int use_atomic) {
    constexpr int NI = kTileOutputs / B;  // output blocks (columns) per CTA
    constexpr int RB = B / 64;            // 16-row blocks per warp (B/4 rows per warp)
    constexpr int CB = NI / 8;            // 8-column blocks per warp
    constexpr int SW_EXTRA = B / 32 + 2;
    constexpr int XW_EXTRA = (B * (NI - 1)) / 32 + 2;
    extern __shared__ __align__(16) uint32_t smb[];
    const int sw = static_cast<int>(kc / 32) + SW_EXTRA;
    uint32_t *S = smb;                              // seed bits from n-1+ka
    uint32_t *X = smb + sw;                         // reversed-key bits from n-1-B*(I0+NI-1)+ka
    uint8_t *par = reinterpret_cast<uint8_t *>(X + static_cast<int>(kc / 32) + XW_EXTRA);

    const uint64_t I0 = uint64_t(blockIdx.x) * NI;
    int64_t klo = static_cast<int64_t>(B * I0) - static_cast<int64_t>(n) + 1;
    klo = (klo >= 0) ? (klo / 32) * 32 : -(((-klo) + 31) / 32) * 32;
    const int64_t khi = static_cast<int64_t>(B * (I0 + NI - 1)) + 1;
    const int64_t ka = klo + static_cast<int64_t>(blockIdx.y) * kc;
    const int64_t kb = ka + kc < khi ? ka + kc : khi;
    const int64_t sbase = static_cast<int64_t>(n) - 1 + ka;
    const int64_t xbase = static_cast<int64_t>(n) - 1 - static_cast<int64_t>(B * (I0 + NI - 1)) + ka;
    stage_bits(S, sw, seed32, seed_words32, sbase, n + m - 1);
    stage_bits(X, static_cast<int>(kc / 32) + XW_EXTRA, xr, xr_words32, xbase, n);
    for (int i = threadIdx.x; i < kTileOutputs; i += blockDim.x) par[i] = 0;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int row0 = warp * (B / 4);
    int acc[RB][CB][4];
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[r][c][e] = 0;

    const int steps = kb > ka ? static_cast<int>((kb - ka + 31) / 32) : 0;
    for (int s = 0; s < steps; ++s) {
        const int k0 = s * 32;
        // A: rows row0 + 16 rb + g (+8), cols k0 + 4t (+16): seed positions row + k
        uint32_t a[2 * RB + 2];
        const int pa0 = row0 + g + k0 + 4 * t;
#pragma unroll
        for (int q = 0; q < 2 * RB + 2; ++q) a[q] = spread(nib(S, pa0 + 8 * q));
        uint32_t bf[CB][2];
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const int pb = B * (NI - 1 - 8 * c - g) + k0 + 4 * t;
            bf[c][0] = spread(nib(X, pb));
            bf[c][1] = spread(nib(X, pb + 16));
        }
#pragma unroll
        for (int r = 0; r < RB; ++r)
#pragma unroll
            for (int c = 0; c < CB; ++c)
                mma_s8(acc[r][c], a[2 * r], a[2 * r + 1], a[2 * r + 2], a[2 * r + 3], bf[c][0],
                       bf[c][1]);
    }
    // parities into par[col * B + row]
#pragma unroll
    for (int r = 0; r < RB; ++r)
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const int row = row0 + 16 * r + g, col = 8 * c + 2 * t;
            par[col * B + row] = acc[r][c][0] & 1;
            par[(col + 1) * B + row] = acc[r][c][1] & 1;
            par[col * B + row + 8] = acc[r][c][2] & 1;
            par[(col + 1) * B + row + 8] = acc[r][c][3] & 1;
        }
    __syncthreads();
    const uint64_t out_words32 = 2 * ceil_div_dev(m, 64);
    for (int w = threadIdx.x; w < kTileOutputs / 32; w += blockDim.x) {
        uint32_t v = 0;
#pragma unroll 8
        for (int i = 0; i < 32; ++i) v |= static_cast<uint32_t>(par[32 * w + i]) << i;
        const uint64_t i0 = uint64_t(B) * I0 + 32 * uint64_t(w);  // output index of bit 0
        const uint64_t gw = i0 >> 5;
        if (gw >= out_words32) continue;
        if (i0 + 32 > m) v = (m > i0) ? (v & ((1u << (m - i0)) - 1u)) : 0u;
        if (use_atomic) {
            if (v) atomicXor(out32 + gw, v);
        } else {
            out32[gw] = v;
        }
    }
}

}  // namespace

int block_plan(uint64_t n, uint64_t m, const pa_opts *o, BlockCfg *c) {
    *c = BlockCfg();
    uint32_t b = (o && o->block_b) ? o->block_b : 128;
    if (b != 128 && b != 256 && b != 512) return PA_ERR_INVALID;
    c->b = b;
    const uint64_t NI = kTileOutputs / b;
    const uint64_t gx = ceil_div(ceil_div(m, b), NI);
    if (gx > 0x7fffffffu) return PA_ERR_UNSUPPORTED;  // checked before narrowing
    c->grid_x = static_cast<uint32_t>(gx);
    const uint64_t klen = n + b * (NI - 1) + 64;  // contraction length per output tile
    const uint64_t target = uint64_t(kNumSMsGB300) * 8 * 4;
    uint64_t kc = ceil_div(klen * c->grid_x, target);
    kc = round_up(kc < 1024 ? 1024 : kc, 32);
    if (kc > 16384) kc = 16384;
    c->kc = kc;
    const uint64_t gy = ceil_div(klen, kc);
    if (gy > 65535) return PA_ERR_UNSUPPORTED;
    c->grid_y = static_cast<uint32_t>(gy);
    c->xr_words = ceil_div(n, 32);
    c->xr_words_pad = round_up(c->xr_words, 4);
    return PA_OK;
}

size_t block_workspace(const BlockCfg &c) { return round_up(c.xr_words_pad * 4, 256); }

template <int B>
static int launch_b(const PlanCfg &cfg, uint32_t *xr, const uint64_t *seed, uint64_t *out,
                    cudaStream_t s, int use_atomic) {
    const BlockCfg &c = cfg.blk;
    constexpr int NI = kTileOutputs / B;
    const size_t smem = (c.kc / 32 + B / 32 + 2 + c.kc / 32 + (B * (NI - 1)) / 32 + 2) * 4 +
                        kTileOutputs;
    if (smem > 48 * 1024)
        PA_CUDA_TRY(cudaFuncSetAttribute(block_mma_kernel<B>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         static_cast<int>(smem)));
    block_mma_kernel<B><<<dim3(c.grid_x, c.grid_y), kBlkThreads, smem, s>>>(
        reinterpret_cast<const uint32_t *>(seed), 2 * ceil_div(cfg.n + cfg.m - 1, 64), xr,
        c.xr_words_pad, cfg.n, cfg.m, static_cast<uint32_t>(c.kc), reinterpret_cast<uint32_t *>(out),
        use_atomic);
    return PA_OK;
}

int block_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
                 const uint64_t *key, uint64_t *out, cudaStream_t s) {
    if (cfg.blk.tc) return block_tc_launch(cfg, ws, hdr, prof, seed, key, out, s);
    const BlockCfg &c = cfg.blk;
    uint32_t *xr = static_cast<uint32_t *>(ws);
    const int use_atomic = c.grid_y > 1;
    // the key reversal also zeroes the output when the key chunks merge by atomicXor
    prof_begin(prof, K_REVERSE_KEY, s);
    reverse_key_launch(key, cfg.n, xr, c.xr_words, c.xr_words_pad, s, use_atomic ? out : nullptr,
                       ceil_div(cfg.m, 64));
    prof_end(prof, s);
    prof_begin(prof, K_BLOCK_MMA, s);
    int rc = PA_OK;
    if (c.b == 128) rc = launch_b<128>(cfg, xr, seed, out, s, use_atomic);
    else if (c.b == 256) rc = launch_b<256>(cfg, xr, seed, out, s, use_atomic);
    else rc = launch_b<512>(cfg, xr, seed, out, s, use_atomic);
    prof_end(prof, s);
    if (rc != PA_OK) return rc;
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace pa
