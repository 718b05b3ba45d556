// Many independent blocks at once (Sec. 3: batches run in parallel on the GPU;
// Sec. 4: later batches wait for resources), plus the autotuner that picks each
// block's path and tile geometry from measured costs.
//
// A batch plan assigns each block a path. All exact-transform blocks of one prime
// field become tiles of ONE persistent launch (ntt_persistent); blocks the tuner
// gives to another path get their own launches. The whole sequence (output zeroing,
// the persistent launch, the other launches) is captured once in a CUDA graph and
// replayed while the stream and the buffers of non-persistent blocks are unchanged;
// block pointers of persistent tiles are read from a device table each run.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "common.cuh"
#include "guard.h"
#include "tiles.cuh"

namespace pa {

// ---------------------------------------------------------------- autotuner

namespace {

constexpr int kTuneLogMin = 8, kTuneLogMax = 22;

struct Tuner {
    bool valid = false;
    double direct = 0;           // s per bit product
    double block[3] = {0, 0, 0};  // s per (m * (n + 8192)), b = 128, 256, 512
    double block_tc = 0;         // tcgen05 FP8: s per (256-block output tile x (n + 32640))
    double fft = 0;              // s per tile of the default FP32 geometry (per unit N log N)
    double ntt[2][kTuneLogMax + 1] = {};  // s per tile of size 2^k, field 0 / 1
    // latency floors of a single plan (one launch sequence, nothing else on the GPU): one
    // standalone tile pair of size 2^k, and small direct and FP8 blocks (n = 2^16, m = 2^13)
    double ntt1[2][kTuneLogMax + 1] = {};
    double direct1 = 0, block_tc1 = 0;
    double launch = 3e-6;        // s per launch
};

std::mutex g_tune_mu;
Tuner g_tuner[64];

__global__ void fill_pattern(uint32_t *p, uint64_t words, uint32_t salt) {
    for (uint64_t i = blockIdx.x * uint64_t(blockDim.x) + threadIdx.x; i < words;
         i += uint64_t(gridDim.x) * blockDim.x) {
        uint32_t z = static_cast<uint32_t>(i) * 0x9E3779B9u + salt;
        z ^= z >> 16;
        z *= 0x85EBCA6Bu;
        z ^= z >> 13;
        p[i] = z;
    }
}

// Time one plan on synthetic bits (best of a few runs after a warm-up).
double time_plan(const PlanCfg &cfg, uint64_t *key, uint64_t *seed, uint64_t *out, cudaStream_t s) {
    void *mem = nullptr;
    if (cudaMalloc(&mem, kHeaderBytes + cfg.ws_bytes) != cudaSuccess) return INFINITY;
    cudaMemset(mem, 0, kHeaderBytes);
    DevHeader *hdr = static_cast<DevHeader *>(mem);
    void *ws = static_cast<char *>(mem) + kHeaderBytes;
    if ((cfg.path == PA_PATH_NTT31 || cfg.path == PA_PATH_NTT64) && ntt_init(cfg, ws) != PA_OK) {
        cudaFree(mem);
        return INFINITY;
    }
    auto run = [&]() -> int {
        switch (cfg.path) {
            case PA_PATH_DIRECT: return direct_launch(cfg, ws, hdr, nullptr, seed, key, out, s);
            case PA_PATH_NTT31:
            case PA_PATH_NTT64: return ntt_launch(cfg, ws, hdr, nullptr, seed, key, out, s);
            case PA_PATH_FFT: return fft_launch(cfg, ws, hdr, nullptr, seed, key, out, s);
            default: return block_launch(cfg, ws, hdr, nullptr, seed, key, out, s);
        }
    };
    // median of five timed runs after a warm-up run (a single fast or slow run must not
    // move the planner's choice)
    double best = INFINITY;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    if (run() == PA_OK && cudaStreamSynchronize(s) == cudaSuccess) {
        double tv[5];
        int got = 0;
        for (int r = 0; r < 5; ++r) {
            cudaEventRecord(a, s);
            if (run() != PA_OK) break;
            cudaEventRecord(b, s);
            if (cudaEventSynchronize(b) != cudaSuccess) break;
            float ms = 0;
            cudaEventElapsedTime(&ms, a, b);
            tv[got++] = ms * 1e-3;
        }
        if (got == 5) {
            std::sort(tv, tv + 5);
            best = tv[2];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaStreamSynchronize(s);
    cudaFree(mem);
    return best;
}

int calibrate(Tuner *t) {
    const uint64_t max_bits = uint64_t(13) << 20;  // key and seed capacity
    uint64_t *key = nullptr, *seed = nullptr, *out = nullptr;
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&key, max_bits / 8 + 64);
    if (e == cudaSuccess) e = cudaMalloc(&seed, 2 * max_bits / 8 + 64);
    if (e == cudaSuccess) e = cudaMalloc(&out, max_bits / 8 + 64);
    if (e != cudaSuccess) {
        cudaFree(key);
        cudaFree(seed);
        cudaFree(out);
        if (s) cudaStreamDestroy(s);
        return cuda_fail(e);
    }
    fill_pattern<<<256, 256, 0, s>>>(reinterpret_cast<uint32_t *>(key), max_bits / 32, 1);
    fill_pattern<<<256, 256, 0, s>>>(reinterpret_cast<uint32_t *>(seed), 2 * max_bits / 32, 2);
    // bring the GPU to its working clock before anything is timed
    {
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        cudaEventRecord(t0, s);
        float ms = 0;
        for (int r = 0; r < 400 && ms < 200.0f; ++r) {
            fill_pattern<<<1024, 256, 0, s>>>(reinterpret_cast<uint32_t *>(seed), 2 * max_bits / 32, 3 + r);
            if ((r & 15) == 15) {
                cudaEventRecord(t1, s);
                cudaEventSynchronize(t1);
                cudaEventElapsedTime(&ms, t0, t1);
            }
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        fill_pattern<<<256, 256, 0, s>>>(reinterpret_cast<uint32_t *>(seed), 2 * max_bits / 32, 2);
    }
    auto tplan = [&](uint64_t n, uint64_t m, const pa_opts &o, PlanCfg *cfg) -> double {
        if (plan_resolve(n, m, &o, cfg) != PA_OK) return INFINITY;
        return time_plan(*cfg, key, seed, out, s);
    };
    PlanCfg cfg;
    pa_opts o;
    memset(&o, 0, sizeof(o));
    o.device = -1;
    o.path = PA_PATH_DIRECT;
    {
        const uint64_t n = uint64_t(1) << 20, m = uint64_t(1) << 13;
        t->direct = tplan(n, m, o, &cfg) / (double(n) * m);
    }
    o.path = PA_PATH_BLOCK_INT8;
    for (int i = 0; i < 3; ++i) {
        o.block_b = 128u << i;
        const uint64_t n = uint64_t(1) << 20, m = uint64_t(1) << 14;
        t->block[i] = tplan(n, m, o, &cfg) / (double(m) * (n + 8192));
    }
    o.block_b = 0;
    o.path = PA_PATH_BLOCK_FP8;
    {
        const uint64_t n = uint64_t(1) << 20, m = uint64_t(1) << 17;
        t->block_tc = tplan(n, m, o, &cfg) / (double(ceil_div(m, 32768)) * double(n + 32640));
        t->block_tc1 = tplan(uint64_t(1) << 16, uint64_t(1) << 13, o, &cfg);
    }
    o.path = PA_PATH_DIRECT;
    t->direct1 = tplan(uint64_t(1) << 16, uint64_t(1) << 13, o, &cfg);
    o.path = PA_PATH_FFT;
    {
        const uint64_t n = uint64_t(1) << 18, m = uint64_t(1) << 13;
        const double tt = tplan(n, m, o, &cfg);
        t->fft = tt / double(cfg.tr.tiles_in * cfg.tr.tiles_out) /
                 (double(uint64_t(1) << cfg.tr.log2n) * (cfg.tr.log2n + 2));
    }
    // Only the 29-bit field is calibrated: with its transform-domain sums grouped below the
    // prime it takes every key length, and a 64-bit butterfly costs about four 32-bit ones,
    // so the tuner never gives a block to the 64-bit field (a caller can still force it).
    for (int k = 0; k <= kTuneLogMax; ++k) t->ntt[1][k] = t->ntt1[1][k] = INFINITY;
    for (int f = 0; f < 1; ++f) {
        o.path = PA_PATH_NTT31;
        for (int k = kTuneLogMin; k <= kTuneLogMax; ++k) {
            const uint64_t N = uint64_t(1) << k, M = N / 4, L = N - M;
            uint64_t tiles = std::max<uint64_t>(4, std::min<uint64_t>(1024, (uint64_t(1) << 24) >> k));
            while (tiles > 1 && L * tiles > max_bits - 64) tiles /= 2;
            o.log2_transform = static_cast<uint32_t>(k);
            o.tile_out = M;
            o.tile_in = L;
            o.fd_mode = 1;  // calibrate standard pairs
            const double tt = tplan(L * tiles, M, o, &cfg);
            t->ntt[f][k] = tt / double(cfg.tr.tiles_in * cfg.tr.tiles_out);
            t->ntt1[f][k] = tplan(L, M, o, &cfg);
        }
        o.log2_transform = 0;
        o.tile_in = o.tile_out = 0;
        o.fd_mode = 0;
    }
    cudaStreamSynchronize(s);
    cudaFree(key);
    cudaFree(seed);
    cudaFree(out);
    cudaStreamDestroy(s);
    t->valid = true;
    return PA_OK;
}

bool load_cache(Tuner *t, const char *path, const char *dev_name) {
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char name[256] = {0};
    bool ok = fgets(name, sizeof(name), f) != nullptr;
    if (ok) {
        name[strcspn(name, "\n")] = 0;
        ok = strcmp(name, dev_name) == 0;
    }
    int version = 0;
    ok = ok && fscanf(f, "v%d", &version) == 1 && version == 3;
    ok = ok && fscanf(f, "%lf %lf %lf %lf %lf %lf %lf %lf", &t->direct, &t->block[0], &t->block[1],
                      &t->block[2], &t->block_tc, &t->fft, &t->direct1, &t->block_tc1) == 8;
    for (int fl = 0; ok && fl < 2; ++fl)
        for (int k = 0; ok && k <= kTuneLogMax; ++k) ok = fscanf(f, "%lf", &t->ntt[fl][k]) == 1;
    for (int fl = 0; ok && fl < 2; ++fl)
        for (int k = 0; ok && k <= kTuneLogMax; ++k) ok = fscanf(f, "%lf", &t->ntt1[fl][k]) == 1;
    fclose(f);
    t->valid = ok;
    return ok;
}

void save_cache(const Tuner &t, const char *path, const char *dev_name) {
    FILE *f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "%s\nv3\n%.6e %.6e %.6e %.6e %.6e %.6e %.6e %.6e\n", dev_name, t.direct, t.block[0],
            t.block[1], t.block[2], t.block_tc, t.fft, t.direct1, t.block_tc1);
    for (int fl = 0; fl < 2; ++fl) {
        for (int k = 0; k <= kTuneLogMax; ++k) fprintf(f, "%.6e ", t.ntt[fl][k]);
        fprintf(f, "\n");
    }
    for (int fl = 0; fl < 2; ++fl) {
        for (int k = 0; k <= kTuneLogMax; ++k) fprintf(f, "%.6e ", t.ntt1[fl][k]);
        fprintf(f, "\n");
    }
    fclose(f);
}

int get_tuner(Tuner *out) {
    int dev = 0;
    PA_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    Tuner &t = g_tuner[dev];
    if (!t.valid) {
        cudaDeviceProp prop;
        PA_CUDA_TRY(cudaGetDeviceProperties(&prop, dev));
        const char *cache = getenv("PA_TUNER_CACHE");
        if (!(cache && load_cache(&t, cache, prop.name))) {
            int rc = calibrate(&t);
            if (rc != PA_OK) return rc;
            if (cache) save_cache(t, cache, prop.name);
        }
    }
    *out = t;
    return PA_OK;
}

// Estimated seconds of one block on each path; fills opts with the best choice.
double best_path(uint64_t n, uint64_t m, const Tuner &t, bool batched, pa_opts *best,
                 uint32_t fd_mode = 0, uint32_t fd_group = 0) {
    memset(best, 0, sizeof(*best));
    best->device = -1;
    double bt = INFINITY;
    auto consider = [&](double tt, const pa_opts &o) {
        if (tt < bt) {
            bt = tt;
            *best = o;
        }
    };
    pa_opts o;
    memset(&o, 0, sizeof(o));
    o.device = -1;
    // a single plan cannot beat the latency of its own launch sequence: floors measured on
    // small blocks (batched blocks share their launches, so no floor applies)
    const auto floor = [batched](double est, double fl) { return batched ? est : std::max(est, fl); };
    o.path = PA_PATH_DIRECT;
    consider(floor(t.direct * double(n) * double(m) + 2 * t.launch, t.direct1), o);
    o.path = PA_PATH_BLOCK_INT8;
    for (int i = 0; i < 3; ++i) {
        o.block_b = 128u << i;
        consider(t.block[i] * double(m) * double(n + 8192) + 2 * t.launch, o);
    }
    o.block_b = 0;
    o.path = PA_PATH_BLOCK_FP8;
    consider(floor(t.block_tc * double(ceil_div(m, 32768)) * double(n + 32640) + 3 * t.launch, t.block_tc1),
             o);
    // FFT path at its usual proven geometry (N = 2^12, L = 1536, M = 2560)
    o.path = PA_PATH_FFT;
    consider(t.fft * double(ceil_div(n, 1536)) * double(ceil_div(m, 2560)) * 4096.0 * 14.0 +
                 t.launch,
             o);
    // transform paths: geometry search with measured per-tile costs; above the calibrated
    // sizes (only multi-output accumulation runs there) a pair's cost is extrapolated from
    // the largest calibrated one as N (log2 N + 6), the geometry model's pair cost
    const auto per_pair = [](const double (&c)[kTuneLogMax + 1], int k) {
        if (k <= kTuneLogMax) return c[k];
        return c[kTuneLogMax] * double(uint64_t(1) << (k - kTuneLogMax)) * double(k + 6) /
               double(kTuneLogMax + 6);
    };
    for (int f = 0; f < 2; ++f) {
        if (!(t.ntt[f][kTuneLogMax] < INFINITY)) continue;  // field not calibrated
        o.path = f == 0 ? PA_PATH_NTT31 : PA_PATH_NTT64;
        for (int k = kTuneLogMin; k <= kLogMax; ++k) {
            const uint64_t N = uint64_t(1) << k;
            const uint64_t mc = round_up(m, 64);
            for (uint64_t div = 1; div <= 256; div *= 2) {
                uint64_t M = div == 1 ? mc : round_up(N / div, 64);
                if (M > mc) M = mc;
                if (M == 0 || M + 32 > N) continue;
                uint64_t L = ((N - M) / 32) * 32;
                if (L > round_up(n, 32)) L = round_up(n, 32);
                uint32_t fd = 0, kgroup = 0;
                uint64_t windows = 0;
                SegChoice seg;  // beyond the resident cap: segmented sums, default sizes
                const double units = ntt_geometry_cost(n, m, f == 0 ? kFieldF29 : kFieldF64,
                                                       static_cast<uint32_t>(k), M, L, fd_mode, fd_group,
                                                       &fd, &windows, &kgroup, &seg);
                const double launches = batched ? 0.0 : 2.0;
                o.log2_transform = static_cast<uint32_t>(k);
                o.tile_out = M;
                o.tile_in = L;
                o.fd_mode = fd_mode;
                o.fd_group = fd_group;
                consider(floor(units * per_pair(t.ntt[f], k) + launches * t.launch, per_pair(t.ntt1[f], k)),
                         o);
            }
        }
        o.log2_transform = 0;
        o.tile_in = o.tile_out = 0;
    }
    return bt;
}

}  // namespace

// Path choice for a single AUTO plan (calibrates on first use on this device).
int tuned_opts(uint64_t n, uint64_t m, pa_opts *out) {
    Tuner t;
    int rc = get_tuner(&t);
    if (rc != PA_OK) return rc;
    best_path(n, m, t, false, out);
    return PA_OK;
}

// ---------------------------------------------------------------- batch zeroing

namespace {
__global__ void batch_zero(const BlockPtrs *__restrict__ blks, const uint32_t *__restrict__ idx) {
    const BlockPtrs b = blks[idx[blockIdx.x]];
    const uint64_t words = 2 * ((b.m + 63) >> 6);
    for (uint64_t w = threadIdx.x; w < words; w += blockDim.x) b.out32[w] = 0u;
}
}  // namespace

}  // namespace pa

using namespace pa;

namespace pa {
// Words per piece of pa_batch_run_host's copies (64 KB).
constexpr uint64_t kCopyPiece = 8192;
// One contiguous copy of 64-bit words (pa_batch_run_host's gather and scatter kernels).
struct CopySeg {
    const uint64_t *src;
    uint64_t *dst;
    uint64_t words;
};
}  // namespace pa

struct pa_batch_s {
    int device = 0;
    std::vector<uint64_t> n, m;
    std::vector<PlanCfg> cfg;
    std::vector<size_t> ws_off;       // per block (non-persistent paths)
    std::vector<uint32_t> in_ntt[kNumFields];  // blocks run by the persistent launches, per field
    NttBatchInfo ntt[kNumFields];
    size_t off_blks = 0, off_idx[kNumFields] = {}, off_ntt[kNumFields] = {}, bytes = 0;
    void *mem = nullptr;
    std::vector<BlockPtrs> hblks;
    bool blks_valid = false;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream the graph is captured on
    cudaStream_t last_stream = nullptr;
    bool graph_ok = false;
    Prof prof;
    uint32_t per_path[8] = {0};
    uint64_t work_items = 0;
    double bound = 0;
    bool eager = false;               // launch without graph capture (serving waves)
    cudaStream_t alloc_stream = nullptr;  // stream-ordered allocation (serving waves)
    // staging for pa_batch_run_host
    void *stage = nullptr;
    std::vector<size_t> st_seed, st_key, st_out;
    size_t stage_bytes = 0;
    pa::CopySeg *segs = nullptr;      // device copy tables: input pieces, then output pieces
    size_t segs_cap = 0;
    std::vector<pa::CopySeg> hsegs;
};

namespace {

DevHeader *batch_hdr(pa_batch_s *b) { return static_cast<DevHeader *>(b->mem); }

// Blocks whose transforms run in the shared persistent launch of their prime field (a
// segmented block runs its own sequence of launches, one per segment, over its own
// workspace).
bool in_persistent(const PlanCfg &c) {
    return (c.path == PA_PATH_NTT31 || c.path == PA_PATH_NTT64) && c.tr.segs.empty();
}

int enqueue_all(pa_batch_s *b, cudaStream_t s) {
    char *base = static_cast<char *>(b->mem);
    const BlockPtrs *dblks = reinterpret_cast<const BlockPtrs *>(base + b->off_blks);
    DevHeader *hdr = batch_hdr(b);
    Prof *prof = b->prof.on ? &b->prof : nullptr;
    for (int f = 0; f < kNumFields; ++f) {
        if (b->in_ntt[f].empty()) continue;
        prof_begin(prof, K_MEMSET, s);
        batch_zero<<<static_cast<unsigned>(b->in_ntt[f].size()), 256, 0, s>>>(
            dblks, reinterpret_cast<const uint32_t *>(base + b->off_idx[f]));
        prof_end(prof, s);
        PA_CUDA_TRY(cudaGetLastError());
        int rc = ntt_batch_launch(b->ntt[f], base + b->off_ntt[f], dblks, &hdr->status, prof, s);
        if (rc != PA_OK) return rc;
    }
    for (size_t i = 0; i < b->cfg.size(); ++i) {
        const PlanCfg &c = b->cfg[i];
        if (in_persistent(c)) continue;
        const BlockPtrs &p = b->hblks[i];
        const uint64_t *seed = reinterpret_cast<const uint64_t *>(p.seed32);
        const uint64_t *key = reinterpret_cast<const uint64_t *>(p.key32);
        uint64_t *out = reinterpret_cast<uint64_t *>(p.out32);
        void *ws = base + b->ws_off[i];
        int rc = PA_OK;
        if (c.path == PA_PATH_DIRECT) rc = direct_launch(c, ws, hdr, prof, seed, key, out, s);
        else if (c.path == PA_PATH_FFT) rc = fft_launch(c, ws, hdr, prof, seed, key, out, s);
        else if (c.path == PA_PATH_NTT31 || c.path == PA_PATH_NTT64)  // segmented block
            rc = ntt_launch(c, ws, hdr, prof, seed, key, out, s);
        else rc = block_launch(c, ws, hdr, prof, seed, key, out, s);
        if (rc != PA_OK) return rc;
    }
    return PA_OK;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

namespace pa {

void batch_free(pa_batch_s *b) {
    if (!b) return;
    if (b->alloc_stream) {
        if (b->mem) cudaFreeAsync(b->mem, b->alloc_stream);
    } else {
        cudaFree(b->mem);
    }
    b->mem = nullptr;
}

int batch_plan_impl(const pa_block *blocks, size_t count, const pa_opts *opts,
                    cudaStream_t alloc_stream, bool eager, pa_batch_s **out) {
    if (!out || !blocks || count == 0 || count > (size_t(1) << 24)) return PA_ERR_INVALID;
    *out = nullptr;
    for (size_t i = 0; i < count; ++i)
        if (!sizes_valid(blocks[i].n, blocks[i].m)) return PA_ERR_INVALID;
    // the batch is freed (device memory and all) on every early return
    const auto release = [](pa_batch_s *x) {
        batch_free(x);
        delete x;
    };
    std::unique_ptr<pa_batch_s, decltype(release)> own(new (std::nothrow) pa_batch_s(), release);
    pa_batch_s *b = own.get();
    if (!b) return PA_ERR_NOMEM;
    b->eager = eager;
    b->alloc_stream = alloc_stream;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) return cuda_fail(e);
    const bool forced = opts && opts->path != PA_PATH_AUTO;
    Tuner t;
    if (!forced) {
        const int rc = get_tuner(&t);
        if (rc != PA_OK) return rc;
    }
    std::vector<BatchBlock> nb[kNumFields];
    size_t off = kHeaderBytes;
    b->off_blks = off;
    off = round_up(off + count * sizeof(BlockPtrs), 256);
    b->cfg.resize(count);
    b->ws_off.assign(count, 0);
    for (size_t i = 0; i < count; ++i) {
        const uint64_t n = blocks[i].n, m = blocks[i].m;
        b->n.push_back(n);
        b->m.push_back(m);
        pa_opts o;
        if (forced) {
            o = *opts;
        } else {
            // the autotuner's choice; a caller's fd_mode and fd_group still apply to NTT
            // blocks
            best_path(n, m, t, true, &o, opts ? opts->fd_mode : 0, opts ? opts->fd_group : 0);
        }
        const int rc = plan_resolve(n, m, &o, &b->cfg[i], false);
        if (rc != PA_OK) return rc;
        const PlanCfg &c = b->cfg[i];
        b->per_path[c.path] += 1;
        if (in_persistent(c)) {
            const int f = c.tr.field;
            BatchBlock bb;
            bb.index = static_cast<uint32_t>(i);
            bb.n = n;
            bb.m = m;
            bb.tr = c.tr;
            nb[f].push_back(bb);
            b->in_ntt[f].push_back(static_cast<uint32_t>(i));
        } else {
            b->ws_off[i] = off;
            off = round_up(off + c.ws_bytes, 256);
            b->work_items += c.path == PA_PATH_FFT ? c.tr.tiles_in * c.tr.tiles_out
                             : c.path == PA_PATH_DIRECT
                                 ? uint64_t(c.direct.grid_x) * c.direct.grid_y
                                 : (c.path == PA_PATH_NTT31 || c.path == PA_PATH_NTT64)
                                       ? [&c] {
                                             uint64_t w = 0;
                                             for (const NttLayout &l : c.tr.segs) w += l.nitems;
                                             return w;
                                         }()
                                       : uint64_t(c.blk.grid_x) * c.blk.grid_y;
            if (c.path == PA_PATH_FFT) b->bound = std::max(b->bound, c.tr.bound);
        }
    }
    for (int f = 0; f < kNumFields; ++f) {
        if (nb[f].empty()) continue;
        const int rc = ntt_batch_build(f, nb[f], opts ? opts->max_slots : 0, &b->ntt[f]);
        if (rc != PA_OK) return rc;
        b->work_items += b->ntt[f].nitems;
        b->off_idx[f] = off;
        off = round_up(off + b->in_ntt[f].size() * sizeof(uint32_t), 256);
        b->off_ntt[f] = off;
        off = round_up(off + b->ntt[f].bytes, 256);
    }
    b->bytes = off;
    cudaStream_t as = alloc_stream;
    e = as ? cudaMallocAsync(&b->mem, b->bytes, as) : cudaMalloc(&b->mem, b->bytes);
    if (e == cudaSuccess)
        e = as ? cudaMemsetAsync(b->mem, 0, kHeaderBytes, as) : cudaMemset(b->mem, 0, kHeaderBytes);
    for (int f = 0; e == cudaSuccess && f < kNumFields; ++f)
        if (!b->in_ntt[f].empty())
            e = cudaMemcpyAsync(static_cast<char *>(b->mem) + b->off_idx[f], b->in_ntt[f].data(),
                                b->in_ntt[f].size() * sizeof(uint32_t), cudaMemcpyHostToDevice, as);
    if (e != cudaSuccess) return cuda_fail(e);
    for (int f = 0; f < kNumFields; ++f) {
        if (b->in_ntt[f].empty()) continue;
        const int rc = ntt_batch_upload(b->ntt[f], static_cast<char *>(b->mem) + b->off_ntt[f], as);
        if (rc != PA_OK) return rc;
    }
    // segmented NTT blocks: their work lists go into their own workspace now (synchronous
    // copies, after the stream-ordered allocation has happened)
    for (size_t i = 0; i < count; ++i) {
        const PlanCfg &c = b->cfg[i];
        if ((c.path != PA_PATH_NTT31 && c.path != PA_PATH_NTT64) || in_persistent(c)) continue;
        if (as) PA_CUDA_TRY(cudaStreamSynchronize(as));
        const int rc = ntt_init(c, static_cast<char *>(b->mem) + b->ws_off[i]);
        if (rc != PA_OK) return rc;
    }
    if (!as) PA_CUDA_TRY(cudaStreamSynchronize(nullptr));
    // root tables of the FFT path are created now, not inside a graph capture
    for (size_t i = 0; i < count; ++i)
        if (b->cfg[i].path == PA_PATH_FFT) {
            const int rc = fft_prepare(b->cfg[i].tr.fp64);
            if (rc != PA_OK) return rc;
        }
    b->hblks.resize(count);
    *out = own.release();
    return PA_OK;
}

// Release a batch. Server-owned batches free their memory in stream order and do not
// synchronise the device; others synchronise their last stream first.
// Copies the words of every segment; CTAs stride over the segments, threads over
// 16-byte vectors where both ends allow it (else words), eight loads in flight per
// thread: the source may be host memory reached over the CPU-GPU link, with a long latency.
__global__ void __launch_bounds__(256) copy_segments(const CopySeg *__restrict__ segs, uint32_t nseg) {
    constexpr int U = 8;
    for (uint32_t sg = blockIdx.x; sg < nseg; sg += gridDim.x) {
        const CopySeg g = segs[sg];
        uint64_t head = 0;  // words copied one by one before the vector part
        const bool vec = ((reinterpret_cast<uintptr_t>(g.src) ^ reinterpret_cast<uintptr_t>(g.dst)) & 15u) == 0;
        if (vec && (reinterpret_cast<uintptr_t>(g.src) & 15u)) head = 1;
        if (head > g.words) head = g.words;
        const uint64_t nv = vec ? (g.words - head) / 2 : 0;  // 16-byte vectors
        const uint4 *vs = reinterpret_cast<const uint4 *>(g.src + head);
        uint4 *vd = reinterpret_cast<uint4 *>(g.dst + head);
        for (uint64_t i = threadIdx.x; i < nv; i += U * uint64_t(blockDim.x)) {
            uint4 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t j = i + u * uint64_t(blockDim.x);
                if (j < nv) v[u] = vs[j];
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t j = i + u * uint64_t(blockDim.x);
                if (j < nv) vd[j] = v[u];
            }
        }
        // the words outside the vector part (all of them when the alignments differ)
        const uint64_t tail0 = head + 2 * nv;
        for (uint64_t w = threadIdx.x; w < head + (g.words - tail0); w += blockDim.x) {
            const uint64_t k = w < head ? w : tail0 + (w - head);
            g.dst[k] = g.src[k];
        }
    }
}

// The device address of page-locked host memory the current device can access (NULL for
// pageable or unknown memory).
void *mapped_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

void batch_destroy_impl(pa_batch_s *b) {
    if (!b) return;
    if (!b->alloc_stream) {
        if (b->last_stream) cudaStreamSynchronize(b->last_stream);
        if (b->cap_stream) cudaStreamSynchronize(b->cap_stream);
    }
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    batch_free(b);
    if (b->stage) cudaFree(b->stage);
    if (b->segs) cudaFree(b->segs);
    prof_free(&b->prof);
    delete b;
}

size_t batch_bytes(const pa_batch_s *b) { return b ? b->bytes : 0; }

}  // namespace pa

extern "C" {

int pa_batch_plan(const pa_block *blocks, size_t count, const pa_opts *opts, pa_batch_t *out) {
    return guarded([&] { return batch_plan_impl(blocks, count, opts, nullptr, false, out); });
}

int pa_batch_run(pa_batch_t b, const pa_block *blocks, size_t count, void *stream, pa_report *rep) {
    return guarded([&] {
        if (!b || !blocks || count != b->cfg.size()) return PA_ERR_INVALID;
        bool changed_other = false, changed_any = !b->blks_valid;
        for (size_t i = 0; i < count; ++i) {
            const pa_block &x = blocks[i];
            if (x.n != b->n[i] || x.m != b->m[i] || !x.seed_bits || !x.key_bits || !x.out_bits)
                return PA_ERR_INVALID;
            if (!aligned16(x.seed_bits) || !aligned16(x.key_bits) || !aligned16(x.out_bits))
                return PA_ERR_ALIGN;
            BlockPtrs p{reinterpret_cast<const uint32_t *>(x.key_bits),
                        reinterpret_cast<const uint32_t *>(x.seed_bits),
                        reinterpret_cast<uint32_t *>(x.out_bits), x.n, x.m};
            BlockPtrs &h = b->hblks[i];
            if (h.key32 != p.key32 || h.seed32 != p.seed32 || h.out32 != p.out32) {
                changed_any = true;
                if (!in_persistent(b->cfg[i])) changed_other = true;
                h = p;
            }
        }
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        if (changed_any) {
            PA_CUDA_TRY(cudaMemcpyAsync(static_cast<char *>(b->mem) + b->off_blks, b->hblks.data(),
                                        count * sizeof(BlockPtrs), cudaMemcpyHostToDevice, s));
            b->blks_valid = true;
        }
        uint32_t replayed = 0;
        if (b->prof.on || b->eager) {
            int rc = enqueue_all(b, s);
            if (rc != PA_OK) return rc;
        } else {
            if (!b->graph_ok || changed_other) {
                if (b->exec) {
                    cudaGraphExecDestroy(b->exec);
                    b->exec = nullptr;
                }
                b->graph_ok = false;
                // capture on a private stream (the caller's may be the legacy default
                // stream, which cannot be captured); the graph is launched on the caller's
                if (!b->cap_stream)
                    PA_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
                cudaGraph_t g = nullptr;
                PA_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
                // the capture ends on every path, an exception in the enqueue included
                int rc = guarded([&] { return enqueue_all(b, b->cap_stream); });
                cudaError_t e = cudaStreamEndCapture(b->cap_stream, &g);
                if (rc != PA_OK) {
                    if (g) cudaGraphDestroy(g);
                    return rc;
                }
                if (e != cudaSuccess) return cuda_fail(e);
                e = cudaGraphInstantiate(&b->exec, g, 0);
                cudaGraphDestroy(g);
                if (e != cudaSuccess) return cuda_fail(e);
                b->graph_ok = true;
            } else {
                replayed = 1;
            }
            PA_CUDA_TRY(cudaGraphLaunch(b->exec, s));
        }
        b->last_stream = s;
        if (rep) {
            PA_CUDA_TRY(cudaStreamSynchronize(s));
            DevHeader h;
            PA_CUDA_TRY(cudaMemcpy(&h, b->mem, sizeof(h), cudaMemcpyDeviceToHost));
            memset(rep, 0, sizeof(*rep));
            memcpy(&rep->max_residual, &h.residual_bits, sizeof(double));
            rep->bound = b->bound;
            for (int i = 0; i < 8; ++i) rep->blocks_per_path[i] = b->per_path[i];
            rep->work_items = b->work_items;
            rep->graph_replayed = replayed;
            if (h.status != 0) {
                int zero = 0;
                cudaMemcpy(b->mem, &zero, sizeof(zero), cudaMemcpyHostToDevice);
                return h.status;
            }
        }
        return PA_OK;
    });
}

namespace {

// Device staging of pa_batch_run_host(_async) (allocated on first use) and the device
// descriptors of the staged blocks; PA_ERR_INVALID if a host block does not match the plan.
int host_stage(pa_batch_s *b, const pa_block *host_blocks, size_t count, std::vector<pa_block> *dev) {
    if (!b->stage) {
        // offsets first (the batch is untouched if a vector cannot grow), then the memory
        std::vector<size_t> seed_off(count), key_off(count), out_off(count);
        size_t off = 0;
        for (size_t i = 0; i < count; ++i) {
            seed_off[i] = off;
            off = round_up(off + ceil_div(b->n[i] + b->m[i] - 1, 64) * 8, 256);
            key_off[i] = off;
            off = round_up(off + ceil_div(b->n[i], 64) * 8, 256);
            out_off[i] = off;
            off = round_up(off + ceil_div(b->m[i], 64) * 8, 256);
        }
        cudaError_t e = cudaMalloc(&b->stage, off);
        if (e != cudaSuccess) {
            b->stage = nullptr;
            return cuda_fail(e);
        }
        b->st_seed = std::move(seed_off);
        b->st_key = std::move(key_off);
        b->st_out = std::move(out_off);
        b->stage_bytes = off;
    }
    char *st = static_cast<char *>(b->stage);
    dev->resize(count);
    for (size_t i = 0; i < count; ++i) {
        const pa_block &h = host_blocks[i];
        if (h.n != b->n[i] || h.m != b->m[i] || !h.seed_bits || !h.key_bits || !h.out_bits)
            return PA_ERR_INVALID;
        (*dev)[i] = {h.n, h.m, reinterpret_cast<const uint64_t *>(st + b->st_seed[i]),
                     reinterpret_cast<const uint64_t *>(st + b->st_key[i]),
                     reinterpret_cast<uint64_t *>(st + b->st_out[i])};
    }
    return PA_OK;
}

}  // namespace

int pa_batch_run_host(pa_batch_t b, const pa_block *host_blocks, size_t count, void *stream,
                      pa_report *rep) {
    return guarded([&] {
        if (!b || !host_blocks || count != b->cfg.size()) return PA_ERR_INVALID;
        std::vector<pa_block> dev;
        const int src = host_stage(b, host_blocks, count, &dev);
        if (src != PA_OK) return src;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        char *st = static_cast<char *>(b->stage);
        // When every host buffer is page-locked and mapped for this device, one gather kernel
        // reads all keys and seeds and one scatter kernel writes all outputs (instead of three
        // copies per block); otherwise one cudaMemcpyAsync per buffer.
        // Copies are cut into pieces of at most kCopyPiece words so that the large keys and
        // seeds spread over many CTAs instead of setting the kernel's duration on one each.
        std::vector<CopySeg> &sg = b->hsegs;
        sg.clear();
        const auto add = [&sg](const uint64_t *src, uint64_t *dst, uint64_t words) {
            for (uint64_t o = 0; o < words; o += kCopyPiece)
                sg.push_back({src + o, dst + o, std::min<uint64_t>(kCopyPiece, words - o)});
        };
        bool mapped = true;
        std::vector<uint64_t *> outs_dev(count, nullptr);
        for (size_t i = 0; i < count && mapped; ++i) {
            const pa_block &h = host_blocks[i];
            void *ds = mapped_host(h.seed_bits), *dk = mapped_host(h.key_bits);
            outs_dev[i] = static_cast<uint64_t *>(mapped_host(h.out_bits));
            mapped = ds && dk && outs_dev[i];
            if (!mapped) break;
            add(static_cast<const uint64_t *>(ds), reinterpret_cast<uint64_t *>(st + b->st_seed[i]),
                ceil_div(h.n + h.m - 1, 64));
            add(static_cast<const uint64_t *>(dk), reinterpret_cast<uint64_t *>(st + b->st_key[i]),
                ceil_div(h.n, 64));
        }
        size_t nin = 0;
        if (mapped) {
            nin = sg.size();
            for (size_t i = 0; i < count; ++i)
                add(reinterpret_cast<const uint64_t *>(st + b->st_out[i]), outs_dev[i], ceil_div(b->m[i], 64));
            if (!b->segs || b->segs_cap < sg.size()) {
                if (b->segs) cudaFree(b->segs);
                b->segs = nullptr;
                cudaError_t e = cudaMalloc(&b->segs, sg.size() * sizeof(CopySeg));
                if (e != cudaSuccess) return cuda_fail(e);
                b->segs_cap = sg.size();
            }
            PA_CUDA_TRY(cudaMemcpyAsync(b->segs, sg.data(), sg.size() * sizeof(CopySeg),
                                        cudaMemcpyHostToDevice, s));
            int sms = kNumSMsGB300;
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
            copy_segments<<<4 * sms, 256, 0, s>>>(b->segs, static_cast<uint32_t>(nin));
            PA_CUDA_TRY(cudaGetLastError());
        } else {
            for (size_t i = 0; i < count; ++i) {
                const pa_block &h = host_blocks[i];
                PA_CUDA_TRY(cudaMemcpyAsync(st + b->st_seed[i], h.seed_bits,
                                            ceil_div(h.n + h.m - 1, 64) * 8, cudaMemcpyHostToDevice, s));
                PA_CUDA_TRY(cudaMemcpyAsync(st + b->st_key[i], h.key_bits, ceil_div(h.n, 64) * 8,
                                            cudaMemcpyHostToDevice, s));
            }
        }
        int rc = pa_batch_run(b, dev.data(), count, stream, nullptr);
        if (rc != PA_OK) return rc;
        if (mapped) {
            copy_segments<<<4 * kNumSMsGB300, 256, 0, s>>>(b->segs + nin, static_cast<uint32_t>(sg.size() - nin));
            PA_CUDA_TRY(cudaGetLastError());
        } else {
            for (size_t i = 0; i < count; ++i)
                PA_CUDA_TRY(cudaMemcpyAsync(host_blocks[i].out_bits, st + b->st_out[i],
                                            ceil_div(b->m[i], 64) * 8, cudaMemcpyDeviceToHost, s));
        }
        PA_CUDA_TRY(cudaStreamSynchronize(s));
        if (rep) {
            DevHeader h;
            PA_CUDA_TRY(cudaMemcpy(&h, b->mem, sizeof(h), cudaMemcpyDeviceToHost));
            memset(rep, 0, sizeof(*rep));
            memcpy(&rep->max_residual, &h.residual_bits, sizeof(double));
            rep->bound = b->bound;
            for (int i = 0; i < 8; ++i) rep->blocks_per_path[i] = b->per_path[i];
            rep->work_items = b->work_items;
            if (h.status != 0) return h.status;
        }
        return PA_OK;
    });
}

int pa_batch_run_host_async(pa_batch_t b, const pa_block *host_blocks, size_t count, void *stream) {
    return guarded([&] {
        if (!b || !host_blocks || count != b->cfg.size()) return PA_ERR_INVALID;
        std::vector<pa_block> dev;
        const int src = host_stage(b, host_blocks, count, &dev);
        if (src != PA_OK) return src;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        char *st = static_cast<char *>(b->stage);
        // copies by the copy engines (no SM time: they overlap kernels of other streams)
        for (size_t i = 0; i < count; ++i) {
            const pa_block &h = host_blocks[i];
            PA_CUDA_TRY(cudaMemcpyAsync(st + b->st_seed[i], h.seed_bits, ceil_div(h.n + h.m - 1, 64) * 8,
                                        cudaMemcpyHostToDevice, s));
            PA_CUDA_TRY(cudaMemcpyAsync(st + b->st_key[i], h.key_bits, ceil_div(h.n, 64) * 8,
                                        cudaMemcpyHostToDevice, s));
        }
        const int rc = pa_batch_run(b, dev.data(), count, stream, nullptr);
        if (rc != PA_OK) return rc;
        for (size_t i = 0; i < count; ++i)
            PA_CUDA_TRY(cudaMemcpyAsync(host_blocks[i].out_bits, st + b->st_out[i], ceil_div(b->m[i], 64) * 8,
                                        cudaMemcpyDeviceToHost, s));
        return PA_OK;
    });
}

int pa_batch_get_report(pa_batch_t b, void *stream, pa_report *rep) {
    if (!b || !rep) return PA_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    DevHeader h;
    PA_CUDA_TRY(cudaMemcpyAsync(&h, b->mem, sizeof(h), cudaMemcpyDeviceToHost, s));
    PA_CUDA_TRY(cudaStreamSynchronize(s));
    memset(rep, 0, sizeof(*rep));
    memcpy(&rep->max_residual, &h.residual_bits, sizeof(double));
    rep->bound = b->bound;
    for (int i = 0; i < 8; ++i) rep->blocks_per_path[i] = b->per_path[i];
    rep->work_items = b->work_items;
    return h.status != 0 ? h.status : PA_OK;
}

void pa_batch_destroy(pa_batch_t b) { batch_destroy_impl(b); }

int pa_batch_profile(pa_batch_t b, int enable) {
    if (!b) return PA_ERR_INVALID;
    return prof_enable(&b->prof, enable);
}

int pa_batch_kernel_times(pa_batch_t b, pa_kernel_time *out, int max, int *count) {
    if (!b || max < 0) return PA_ERR_INVALID;
    return prof_collect(&b->prof, out, max, count);
}

int pa_batch_describe(pa_batch_t b, pa_plan_desc *out, size_t count) {
    if (!b || !out || count != b->cfg.size()) return PA_ERR_INVALID;
    for (size_t i = 0; i < count; ++i) fill_desc(b->cfg[i], &out[i]);
    return PA_OK;
}

// One-shot: the batch plan is cached for the last shape list (per thread).
int pa_hash_batched(const pa_block *blocks, size_t count, void *stream, pa_report *rep) {
    return guarded([&] {
        static thread_local pa_batch_s *cached = nullptr;
        static thread_local std::vector<uint64_t> shape;
        if (!blocks || count == 0) return PA_ERR_INVALID;
        std::vector<uint64_t> sh;
        sh.reserve(2 * count);
        for (size_t i = 0; i < count; ++i) {
            sh.push_back(blocks[i].n);
            sh.push_back(blocks[i].m);
        }
        int dev = 0;
        PA_CUDA_TRY(cudaGetDevice(&dev));
        if (!cached || sh != shape || cached->device != dev) {
            if (cached) pa_batch_destroy(cached);
            cached = nullptr;
            int rc = pa_batch_plan(blocks, count, nullptr, &cached);
            if (rc != PA_OK) return rc;
            shape = sh;
        }
        return pa_batch_run(cached, blocks, count, stream, rep);
    });
}

}  // extern "C"
