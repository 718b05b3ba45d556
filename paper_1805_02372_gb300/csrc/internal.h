// Internal declarations of the Toeplitz-hash library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "../../include/pa.h"

struct pa_batch_s;

namespace pa {

constexpr int kNumSMsGB300 = 152;

// ---- direct path (bit-packed AND + popcount) ----
struct DirectCfg {
    uint32_t kc = 0;            // 32-bit key words per CTA
    uint64_t key_words32 = 0;   // ceil(n/32)
    uint64_t key_words32_pad = 0;  // padded to a multiple of kc
    uint32_t grid_x = 0, grid_y = 0;
};

// ---- transform paths (NTT over a prime field, FP FFT) ----
// Prime fields of the NTT paths: PA_PATH_NTT64 runs modulo 2^64 - 2^32 + 1; PA_PATH_NTT31
// by default modulo 5*2^25 + 1 when n is below it and 7*2^26 + 1 otherwise (both lazily
// reduced; transform-domain sums grouped below the prime), or 15*2^27 + 1 on request.
constexpr int kFieldF31 = 0, kFieldF64 = 1, kFieldF29 = 2, kFieldF28 = 3, kNumFields = 4;
constexpr uint64_t kPrimeF28 = 167772161ull, kPrimeF29 = 469762049ull, kPrimeF31 = 2013265921ull;

// Workspace layout and launch shape of one persistent NTT launch (see ntt.cu).
struct NttLayout {
    int field = 0;         // kFieldF31 / kFieldF64 / kFieldF29 / kFieldF28
    uint64_t ntiles = 0, nitems = 0, nfd = 0;
    uint32_t slots = 1;    // spectra slots of standard tiles, reused round-robin
    size_t smem = 0;
    size_t off_tiles = 0, off_items = 0, off_fd = 0, off_wmap = 0, off_counters = 0;
    size_t counter_bytes = 0, off_spec = 0;
    size_t bytes = 0;      // workspace bytes
};

struct TransformCfg {
    uint32_t log2n = 0;          // transform size N = 2^log2n
    uint64_t L = 0, M = 0;       // key tile and output tile lengths
    uint64_t tiles_in = 0, tiles_out = 0;
    uint32_t delta = 0;          // extra window shift so output tiles start on 32-bit words
    uint32_t passes = 0;         // NTT: global passes
    uint32_t radix_log2[4] = {0, 0, 0, 0};
    uint32_t fp64 = 0;           // FFT: FP64 butterflies
    double bound = 0.0;          // FFT: proven rounding bound
    int field = 0;               // NTT: kFieldF31 / kFieldF64 / kFieldF29 / kFieldF28
    uint32_t fd = 0;             // NTT: transform-domain accumulation over key tiles
    uint64_t windows = 0;        // NTT with fd: distinct seed-window spectra
    uint32_t kgroup = 0;         // NTT with fd = 1: key tiles per transform-domain sum (the
                                 // counts of a sum stay below the prime); 0 = all of them
    uint32_t outer_logT = 0;     // NTT with fd = 1 and equal tiles: the sums of each group are
    uint32_t outer_slice = 0;    // convolutions over the tile index, computed with 2^outer_logT-
                                 // point transforms for slices of outer_slice output tiles
                                 // (0 = direct sums)
    uint32_t seg_in = 0;         // NTT with fd = 1, segmented: key tiles per segment and
    uint32_t seg_out = 0;        // output tiles per slice (0 = everything resident at once);
                                 // each (slice, segment) is one persistent launch over one
                                 // shared spectra workspace, run in order
    NttLayout lay;               // NTT single-block plans: their persistent launch (segmented:
                                 // lay.bytes is the whole workspace)
    std::vector<NttLayout> segs; // segmented plans: one launch layout per (slice, segment)
    std::vector<size_t> seg_base;  // workspace offset of each segment's tables
};

// ---- block-Toeplitz tensor-core path ----
struct BlockCfg {
    uint32_t b = 0;              // tile edge (rows of each T_d)
    uint64_t kc = 0;             // contraction positions per CTA (multiple of 32)
    uint32_t grid_x = 0, grid_y = 0;
    uint64_t xr_words = 0, xr_words_pad = 0;  // reversed key in the workspace
    uint32_t tc = 0;             // 1: tcgen05 FP8 kernel (block_tc.cu), kc = chunk per CTA
};

struct PlanCfg {
    uint64_t n = 0, m = 0;
    int path = PA_PATH_DIRECT;
    DirectCfg direct;
    TransformCfg tr;
    BlockCfg blk;
    size_t ws_bytes = 0;         // workspace excluding the status header
    uint32_t kernels = 0;
};

// Autotuner: the measured-cost choice of path and tile geometry for one block
// (calibrates by timing each path on the current device on first use).
int tuned_opts(uint64_t n, uint64_t m, pa_opts *out);

// Host-only planning (no GPU calls).
// layout = false: NTT plans skip their single-block work-list layout (a batch builds its
// own combined list; segmented blocks still get theirs).
int plan_resolve(uint64_t n, uint64_t m, const pa_opts *o, PlanCfg *cfg, bool layout = true);
void fill_desc(const PlanCfg &cfg, pa_plan_desc *d);

// Workspace header kept at the start of every plan's device workspace.
struct DevHeader {
    int status;
    int pad;
    unsigned long long residual_bits;  // max |v - rint(v)| as the bit pattern of a double >= 0
};
constexpr size_t kHeaderBytes = 256;

// ---- per-kernel CUDA-event timing (pa_plan_profile / pa_batch_profile) ----
enum KernelId {
    K_REVERSE_KEY = 0,
    K_DIRECT,
    K_FFT_TILE,
    K_BLOCK_MMA,
    K_BATCH_PERSISTENT,
    K_MEMSET,
    K_BLOCK_TC,
    K_NUM_KERNELS
};
const char *kernel_name(int kid);

struct ProfRec {
    int kid;
    cudaEvent_t a, b;
};
struct Prof {
    bool on = false;
    ProfRec *recs = nullptr;
    size_t cap = 0, used = 0;
    int open_kid = -1;
};
// Record an event pair around one launch when profiling is on (no-ops otherwise).
void prof_begin(Prof *p, int kid, cudaStream_t s);
void prof_end(Prof *p, cudaStream_t s);
int prof_enable(Prof *p, int enable);
int prof_collect(Prof *p, pa_kernel_time *out, int max, int *count);
void prof_free(Prof *p);

// Launchers (enqueue on stream; return PA_OK or PA_ERR_CUDA).
int direct_plan(uint64_t n, uint64_t m, DirectCfg *c);
// xr[q] bit c = x[n-1-32q-c] for q < words, zero up to words_pad; the same launch zeroes
// zero_words 64-bit words at `zero` when it is not null.
void reverse_key_launch(const uint64_t *key, uint64_t n, uint32_t *xr, uint64_t words,
                        uint64_t words_pad, cudaStream_t s, uint64_t *zero = nullptr,
                        uint64_t zero_words = 0);
size_t direct_workspace(const DirectCfg &c);
int direct_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
                  const uint64_t *key, uint64_t *out, cudaStream_t s);

// Block-Toeplitz contraction on tcgen05 (FP8 operands, FP32 accumulation in TMEM).
int block_tc_plan(uint64_t n, uint64_t m, const pa_opts *o, BlockCfg *c);
int block_tc_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
                    const uint64_t *key, uint64_t *out, cudaStream_t s);

// Transform sizes of the exact path: standard tile pairs and streamed blocks up to 2^22,
// multi-output transform-domain accumulation up to 2^23.
constexpr int kLogMax = 23;
constexpr int kLogMaxStd = 22;

int ntt_plan(uint64_t n, uint64_t m, int path, const pa_opts *o, TransformCfg *c);
// Modelled cost of a tile geometry over prime field `field` in units of one standard tile
// pair of size 2^k (+inf if invalid); *fd / *windows / *kgroup: whether transform-domain
// accumulation is used, its window spectra and key tiles per sum (fd_group > 0 caps it).
// Geometries whose resident spectra exceed the accumulation cap run segmented (*seg_in key
// tiles per segment, *seg_out output tiles per slice) within seg_cap bytes of spectra;
// seg_in_force / seg_out_force fix the segment sizes (0 = choose).
struct SegChoice {
    uint64_t seg_cap = 0;          // bytes of spectra a segmented plan may hold (0 = default)
    uint32_t seg_in_force = 0, seg_out_force = 0;
    uint32_t seg_in = 0, seg_out = 0;  // out: the choice (0 = not segmented)
    uint32_t outer_mode = 0;       // outer convolutions for the sums: 0 when cheaper, 1 never,
                                   // 2 whenever possible
    uint32_t outer_logT = 0, outer_slice = 0;  // out: the choice (0 = direct sums)
};
double ntt_geometry_cost(uint64_t n, uint64_t m, int field, uint32_t k, uint64_t M, uint64_t L,
                         uint32_t fd_mode, uint32_t fd_group, uint32_t *fd, uint64_t *windows,
                         uint32_t *kgroup, SegChoice *seg = nullptr);
// Lays out the single-block plan's persistent launch (fills c->lay; host only).
int ntt_layout(uint64_t n, uint64_t m, int path, TransformCfg *c);
int ntt_init(const PlanCfg &cfg, void *ws);  // uploads the work list, builds root tables
int ntt_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
               const uint64_t *key, uint64_t *out, cudaStream_t s);

int fft_plan(uint64_t n, uint64_t m, const pa_opts *o, TransformCfg *c);
int fft_prepare(int fp64);  // creates the twiddle table (outside any graph capture)
size_t fft_workspace(const TransformCfg &c);
int fft_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
               const uint64_t *key, uint64_t *out, cudaStream_t s);

int block_plan(uint64_t n, uint64_t m, const pa_opts *o, BlockCfg *c);
size_t block_workspace(const BlockCfg &c);
int block_launch(const PlanCfg &cfg, void *ws, DevHeader *hdr, Prof *prof, const uint64_t *seed,
                 const uint64_t *key, uint64_t *out, cudaStream_t s);

// ---- batches of transform blocks in one persistent launch ----
struct BatchBlock {
    uint32_t index;        // position in the batch (BlockPtrs table index)
    uint64_t n, m;
    TransformCfg tr;
    // fd blocks: the output tiles [I0, I1) and key tiles [J0, J1) this work list covers
    // (I1 = J1 = 0: all of them); a segment of a segmented plan
    uint64_t I0 = 0, I1 = 0, J0 = 0, J1 = 0;
};
struct NttBatchInfo : NttLayout {
    std::vector<unsigned char> host_tiles, host_fd;
    std::vector<uint64_t> host_items;
    std::vector<uint32_t> host_wmap;
};
int ntt_batch_build(int field, const std::vector<BatchBlock> &blocks, uint32_t max_slots,
                    NttBatchInfo *info);
// host tables are copied on stream s (kept alive by info until the copy ran)
int ntt_batch_upload(const NttBatchInfo &info, void *ws, cudaStream_t s);
// blks: device array of the batch's BlockPtrs (see tiles.cuh)
int ntt_batch_launch(const NttBatchInfo &info, void *ws, const void *blks, int *status, Prof *prof,
                     cudaStream_t s);

// Batch plans for the serving engine: alloc_stream != nullptr allocates and frees in
// stream order on it (no device-wide synchronisation); eager = no graph capture.
int batch_plan_impl(const pa_block *blocks, size_t count, const pa_opts *opts,
                    cudaStream_t alloc_stream, bool eager, pa_batch_s **out);
void batch_destroy_impl(pa_batch_s *b);
size_t batch_bytes(const pa_batch_s *b);

// Records a CUDA error for pa_last_cuda_error and maps it to a status.
int cuda_fail(cudaError_t e);
#define PA_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) return ::pa::cuda_fail(_e); \
    } while (0)

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }
inline uint64_t round_up(uint64_t a, uint64_t b) { return ceil_div(a, b) * b; }
inline uint32_t log2_ceil(uint64_t v) {
    uint32_t k = 0;
    while ((uint64_t(1) << k) < v) ++k;
    return k;
}

}  // namespace pa
