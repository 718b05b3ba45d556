// Block-Toeplitz path on the 5th-generation tensor cores (tcgen05): the one dense form
// of the hash, Y[:, I] = sum_d T_d X[:, I-d] with 128 x 128 Toeplitz tiles
// T_d[a][c] = s[n-1+128d+a-c] (the row split of Eq. Ti / Eq. Tij taken down to tiles of
// 128 rows), multiplied with kind::f8f6f4 MMAs accumulating in tensor memory, then mod 2.
//
// As a GEMM (the same contraction as block.cu): C[a][I] = sum_k A[a][k] B[I][k] with
//   A[a][k] = s[n-1+a+k]          (Hankel: row a+1 is row a shifted by one position)
//   B[I][k] = x[128 I - k]         (the reversed key read at stride 128)
// and y[128 I + a] = C[a][I] mod 2. Bits become e4m3 values 0 or 2^-6 (byte 0x08), so a
// product is 0 or 2^-12 and C[a][I] = count * 2^-12 exactly: a CTA's contraction chunk
// is at most 2^15 positions, so every partial sum is a multiple of 2^-12 below 8, which
// FP32 (24-bit significand) holds exactly whatever the order of additions.
//
// CTA (256 threads, two per SM): output blocks I0 .. I0+255 (128 x 256 outputs, the MMA
// shape M = 128, N = 256, FP32 accumulator in 256 TMEM columns) and one chunk of the
// contraction; chunks are XOR-merged into the output (Eq. finalkey). The chunk advances
// in stages of 128 positions (4 MMAs of K = 32); one thread issues the MMAs and commits
// them to an mbarrier.
//
// Both operands are Toeplitz/Hankel, and both layouts exploit it (K-major, no swizzle:
// core matrices of 8 rows x 16 bytes).
//   B (key): with the columns in reverse order (MMA column r' is block I0 + 255 - r'),
//      column r' of stage s holds window positions 128 (r' + s) + [0, 128): stage s + 1
//      is stage s moved by one column. The expanded key window is stored once as a ring
//      of 16-byte row pieces per K core (piece R of core c at c * 16 Rtot + 16 R, rows
//      at 16 bytes, row groups at 128, K cores at 16 Rtot), and the descriptor of stage
//      s starts 16 s bytes in. The whole key side is expanded once per CTA.
//   A (seed): row a, bytes [16c, 16c+16) hold seed positions a + 16c + [0, 16); with
//      a = 8g + i that is position 8(g + 2c) + i + [0, 16), which depends on (g, c) only
//      through u = g + 2c. So core (g, c) is stored once per u ("chunk" u: rows i = 0..7
//      of 16 bytes at u*128 + 16i) and the descriptor steps 128 bytes per row group and
//      256 per K core: 30 chunks (3.75 KB) per stage, double-buffered; all threads
//      expand the next stage's chunks while the tensor core runs the current stage.
#include <string.h>

#include "common.cuh"

namespace pa {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;           // rows a (tile edge b)
constexpr int kTcN = 256;           // output blocks I per CTA
constexpr int kTcStage = 128;       // contraction positions per stage
constexpr int kTcAChunks = 30;      // u = g + 2c, g < 16, c < 8
constexpr int kTcABytes = 4096;
constexpr int kTcMaxChunk = 32768;  // contraction positions per CTA (counts < 2^15)
constexpr int kTcMaxStages = kTcMaxChunk / kTcStage;
constexpr int kTcMaxRows = kTcN + kTcMaxStages;             // key ring rows (Rtot)
constexpr int kTcSeedWords = 4 * kTcMaxStages + 8;          // staged seed words
constexpr size_t kTcUsed = 2 * kTcABytes + 8 * 16 * kTcMaxRows + 4 * kTcSeedWords;
// Dynamic shared memory: A[2] | key ring | seed window, padded so that at most two CTAs
// (2 x 256 TMEM columns) are resident on an SM.
constexpr size_t kTcSmem = kTcUsed > 80 * 1024 ? kTcUsed : 80 * 1024;
static_assert(3 * kTcSmem > 228 * 1024, "three CTAs per SM would oversubscribe TMEM");

// Instruction descriptor, kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B = E4M3 (bits 7-9,
// 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28.
constexpr uint32_t kTcIdesc = (1u << 4) | (uint32_t(kTcN >> 3) << 17) | (uint32_t(kTcM >> 4) << 24);

// Shared-memory matrix descriptor, no swizzle: start address >> 4 (bits 0-13), leading
// (K-direction core) byte offset >> 4 (16-29), stride (8-row group) byte offset >> 4
// (32-45), the fixed version bit 46.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(lbo >> 4) << 16) |
           (uint64_t(sbo >> 4) << 32) | (uint64_t(1) << 46);
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kTcIdesc), "r"(acc)
        : "memory");
}

// Arrives on bar once every MMA this thread issued so far has completed.
__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 16 bits -> 16 e4m3 bytes: bit t of v becomes byte t, 0x00 or 0x08 (= 2^-6). The four
// shifted copies of a nibble (multiplier 0x01020408) occupy disjoint bit ranges, so there
// are no carries, and bit t of the nibble lands on bit 3 of byte t.
__device__ __forceinline__ uint4 expand16(uint32_t v) {
    uint4 r;
    r.x = ((v & 0xFu) * 0x01020408u) & 0x08080808u;
    r.y = (((v >> 4) & 0xFu) * 0x01020408u) & 0x08080808u;
    r.z = (((v >> 8) & 0xFu) * 0x01020408u) & 0x08080808u;
    r.w = (((v >> 12) & 0xFu) * 0x01020408u) & 0x08080808u;
    return r;
}

__device__ __forceinline__ void sts128(uint32_t addr, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

// Bounded wait for the completion of the mbarrier phase with this parity (no status write).
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, uint64_t limit_ns = kWaitNs) {
    return mbar_wait_for(bar, parity, limit_ns);
}

// grid.x: contraction chunks of `chunk` positions; grid.y: output tiles of 256 blocks.
__global__ void __launch_bounds__(kTcThreads, 2) block_tc_kernel(
    const uint32_t *__restrict__ seed32, uint64_t seed_words32, const uint32_t *__restrict__ xr,
    uint64_t xr_words32, uint64_t n, uint64_t m, uint32_t chunk, uint32_t *__restrict__ out32,
    int *status, unsigned long long *residual_bits) {
    extern __shared__ __align__(1024) unsigned char smt[];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint64_t I0 = uint64_t(blockIdx.y) * kTcN;
    const uint64_t klen = n + uint64_t(kTcM) * (kTcN - 1);  // contraction length of a tile
    const uint64_t kdone = uint64_t(blockIdx.x) * chunk;
    const uint64_t kmine = klen - kdone < chunk ? klen - kdone : chunk;
    const int S = static_cast<int>((kmine + kTcStage - 1) / kTcStage);

    const int Rtot = kTcN + S;                 // key ring rows
    const uint32_t lbo_b = 16u * static_cast<uint32_t>(Rtot);
    unsigned char *A = smt;
    unsigned char *Bring = smt + 2 * kTcABytes;
    uint32_t *SW = reinterpret_cast<uint32_t *>(Bring + 8 * 16 * kTcMaxRows);

    // Key ring: row R holds reversed-key window positions 128 R + [0, 128), window start
    // xw0 = kdone - 128 * 255 (tile independent): xr words w0 + 4R .. + 3.
    {
        const int64_t w0 = static_cast<int64_t>(kdone / 32) - 4 * (kTcN - 1);
        const uint32_t ring = smem_addr(Bring);
        for (int R = tid; R < Rtot; R += kTcThreads) {
            const int64_t g = w0 + 4 * R;
            uint32_t ws[4];
            if (g >= 0 && static_cast<uint64_t>(g) + 4 <= xr_words32) {
                const uint4 v = __ldg(reinterpret_cast<const uint4 *>(xr + g));
                ws[0] = v.x, ws[1] = v.y, ws[2] = v.z, ws[3] = v.w;
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    ws[e] = (g + e >= 0 && static_cast<uint64_t>(g + e) < xr_words32) ? __ldg(xr + g + e) : 0u;
            }
#pragma unroll
            for (int c = 0; c < 8; ++c)
                sts128(ring + c * lbo_b + 16 * R, expand16((ws[c >> 1] >> (16 * (c & 1))) & 0xFFFFu));
        }
    }
    // Seed window: word w holds seed bits [sw0 + 32 w, +32), sw0 = 128 I0 + kdone; bits at
    // positions >= n + m - 1 read as 0.
    {
        const uint64_t sl = n + m - 1;
        const uint64_t w0 = (uint64_t(kTcM) * I0 + kdone) / 32;
        const int nw = 4 * S + 8;
        for (int w = tid; w < nw; w += kTcThreads) {
            const uint64_t g = w0 + w;
            uint32_t v = 0;
            if (g < seed_words32 && 32 * g < sl) {
                v = __ldg(seed32 + g);
                if (32 * g + 32 > sl) v &= (1u << (sl - 32 * g)) - 1u;
            }
            SW[w] = v;
        }
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_barrier_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(kTcN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    const uint32_t a_base = smem_addr(A), b_base = smem_addr(Bring);
    int issued = 0;  // stages whose MMAs were issued and committed
    bool bad = false;
    for (int s = 0; s < S; ++s) {
        const int buf = s & 1;
        if (s >= 2) bad = !tc_wait(&bar[buf], ((s - 2) >> 1) & 1);
        if (!bad) {
            // A: chunk u = tid >> 3, row i = tid & 7: seed positions 128 s + 8u + i = 128 s + tid
            if (tid < kTcAChunks * 8) {
                const int q = kTcStage * s + tid;
                const uint32_t v = __funnelshift_r(SW[q >> 5], SW[(q >> 5) + 1], q & 31);
                sts128(a_base + buf * kTcABytes + 16 * tid, expand16(v & 0xFFFFu));
            }
        }
        fence_proxy_async_smem();
        if (__syncthreads_or(bad)) break;
        if (tid == 0) {
            tc_fence_after();
#pragma unroll
            for (int kk = 0; kk < kTcStage / 32; ++kk) {
                const uint64_t ad = smem_desc(a_base + buf * kTcABytes + kk * 512, 256, 128);
                const uint64_t bd = smem_desc(b_base + 16 * s + 2 * kk * lbo_b, lbo_b, 128);
                tc_mma(tmem, ad, bd, (s > 0 || kk > 0) ? 1u : 0u);
            }
            tc_commit(&bar[buf]);
        }
        issued = s + 1;
    }
    // Wait for the last committed stage (it covers every earlier MMA).
    bool ok = !bad;
    if (issued > 0) {
        const int last = issued - 1;
        if (!tc_wait(&bar[last & 1], (last >> 1) & 1, bad ? kDrainNs : kWaitNs)) ok = false;
    }
    if (__syncthreads_or(!ok) || issued == 0) {
        if (tid == 0 && (bad || issued > 0)) set_status(status, PA_ERR_TIMEOUT);
    } else {
        tc_fence_after();
        // Epilogue: warp w reads TMEM lanes 32 (w & 3) + lane (row a) and columns
        // [128 (w >> 2), +128) (column r' is block I = 255 - r'); a ballot over the warp's
        // 32 rows gives one output word per block, bits 128 (I0 + I) + 32 (w & 3) + [0, 32).
        const int q = warp & 3;
        const uint64_t out_words32 = 2 * ceil_div_dev(m, 64);
        float rmax = 0.0f;  // |4096 acc - rint|: 0 whenever the sums are exact, as proven
        for (int c0 = 128 * (warp >> 2); c0 < 128 * (warp >> 2) + 128; c0 += 32) {
            uint32_t mine = 0;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                uint32_t v[16];
                tc_ld16(tmem + (uint32_t(32 * q) << 16) + c0 + 16 * h, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float x = __uint_as_float(v[j]) * 4096.0f;
                    rmax = fmaxf(rmax, fabsf(x - rintf(x)));
                    const uint32_t cnt = __float2uint_rn(x);
                    const uint32_t word = __ballot_sync(0xFFFFFFFFu, cnt & 1u);
                    if (lane == 16 * h + j) mine = word;
                }
            }
            const uint64_t bit0 = uint64_t(kTcM) * (I0 + (kTcN - 1) - (c0 + lane)) + 32 * q;
            const uint64_t gw = bit0 >> 5;
            if (bit0 < m && gw < out_words32) {
                if (bit0 + 32 > m) mine &= (1u << (m - bit0)) - 1u;
                if (mine) atomicXor(out32 + gw, mine);
            }
        }
        // the worst pre-rounding residual, reported per run (pa_last_residual); one atomic
        // per warp only when it is not zero
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) rmax = fmaxf(rmax, __shfl_xor_sync(0xFFFFFFFFu, rmax, o));
        if (lane == 0 && rmax > 0.0f)
            atomicMax(residual_bits, static_cast<unsigned long long>(__double_as_longlong(double(rmax))));
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcN)
                     : "memory");
    }
}

}  // namespace

int block_tc_plan(uint64_t n, uint64_t m, const pa_opts *o, BlockCfg *c) {
    *c = BlockCfg();
    if (o && o->block_b && o->block_b != static_cast<uint32_t>(kTcM)) return PA_ERR_INVALID;
    c->b = kTcM;
    c->tc = 1;
    const uint64_t tiles = ceil_div(m, uint64_t(kTcM) * kTcN);
    const uint64_t klen = n + uint64_t(kTcM) * (kTcN - 1);
    // about four waves of two CTAs per SM, chunks of 1024 .. 32768 positions
    const uint64_t target = uint64_t(kNumSMsGB300) * 2 * 4;
    uint64_t chunk = round_up(ceil_div(klen * tiles, target), kTcStage);
    if (chunk < 1024) chunk = 1024;
    if (chunk > static_cast<uint64_t>(kTcMaxChunk)) chunk = kTcMaxChunk;
    if (o && o->tile_in) {  // caller's chunk: a multiple of the stage, at most kTcMaxChunk
        if (o->tile_in % kTcStage || o->tile_in > static_cast<uint64_t>(kTcMaxChunk))
            return PA_ERR_INVALID;
        chunk = o->tile_in;
    }
    const uint64_t chunks = ceil_div(klen, chunk);
    if (tiles > 65535 || chunks > 0x7fffffffu) return PA_ERR_UNSUPPORTED;
    c->kc = chunk;
    c->grid_x = static_cast<uint32_t>(chunks);
    c->grid_y = static_cast<uint32_t>(tiles);
    c->xr_words = ceil_div(n, 32);
    c->xr_words_pad = round_up(c->xr_words, 4);
    return PA_OK;
}

int block_tc_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
                    const uint64_t *key, uint64_t *out, cudaStream_t s) {
    const BlockCfg &c = cfg.blk;
    uint32_t *xr = static_cast<uint32_t *>(ws);
    // the key reversal also zeroes the output (the contraction merges by atomicXor)
    prof_begin(prof, K_REVERSE_KEY, s);
    reverse_key_launch(key, cfg.n, xr, c.xr_words, c.xr_words_pad, s, out, ceil_div(cfg.m, 64));
    prof_end(prof, s);
    PA_CUDA_TRY(cudaFuncSetAttribute(block_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     static_cast<int>(kTcSmem)));
    prof_begin(prof, K_BLOCK_TC, s);
    block_tc_kernel<<<dim3(c.grid_x, c.grid_y), kTcThreads, kTcSmem, s>>>(
        reinterpret_cast<const uint32_t *>(seed), 2 * ceil_div(cfg.n + cfg.m - 1, 64), xr, c.xr_words,
        cfg.n, cfg.m, static_cast<uint32_t>(c.kc), reinterpret_cast<uint32_t *>(out), &hdr->status,
        &hdr->residual_bits);
    prof_end(prof, s);
    PA_CUDA_TRY(cudaGetLastError());
    return PA_OK;
}

}  // namespace pa
