// C ABI of the Toeplitz-hash library: planning, single-block hashing, status.
// Every entry point returns a pa_status; no exception crosses the interface (guard.h).
#include <algorithm>
#include <new>
#include <string.h>

#include "guard.h"
#include "internal.h"
#include "ntt_defs.cuh"

namespace pa {

static thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e) {
    g_last_cuda_error = static_cast<int>(e);
    if (e == cudaErrorMemoryAllocation) return PA_ERR_NOMEM;
    return PA_ERR_CUDA;
}

// Standard tile pairs (no transform-domain sums) a plan may lay out, and work items
// their persistent launch may list (2^28 items: 2 GiB of work list on host and device).
constexpr uint64_t kStdMaxPairs = uint64_t(1) << 22;
constexpr uint64_t kStdMaxItems = uint64_t(1) << 28;

// Work items of a standard NTT plan: one per one-CTA tile pair; above 2^kLogSmallMax
// points, per pair two forward pass-1 sweeps (key tile and seed window) and one inverse
// of g1 column groups each, and g2 row groups of pass 2 (the work list's layout).
static double std_items(const TransformCfg &t) {
    const double pairs = double(t.tiles_in) * double(t.tiles_out);
    if (t.log2n <= static_cast<uint32_t>(kLogSmallMax)) return pairs;
    int logR1 = 0, logR2 = 0, logC1 = 0, logC2 = 0;
    split_r(static_cast<int>(t.log2n), &logR1, &logR2);
    pass_columns(static_cast<int>(t.log2n), t.field == kFieldF64 ? 8 : 4, &logC1, &logC2);
    const double g1 = double(uint64_t(1) << (t.log2n - logR1 - logC1));
    const double g2 = double(uint64_t(1) << (logR1 - logC2));
    return pairs * (3.0 * g1 + g2);
}

int plan_resolve(uint64_t n, uint64_t m, const pa_opts *o, PlanCfg *cfg, bool layout) {
    if (!cfg || !sizes_valid(n, m)) return PA_ERR_INVALID;
    *cfg = PlanCfg();
    cfg->n = n;
    cfg->m = m;
    int path = o ? o->path : PA_PATH_AUTO;
    if (path < PA_PATH_AUTO || path > PA_PATH_BLOCK_FP8) return PA_ERR_INVALID;
    if (path == PA_PATH_AUTO) {
        // Host-only rule (pa_plan_ex uses the autotuner's measured costs instead): the
        // direct kernel while m*n is small; beyond, the exact NTT over the 28- or 29-bit prime
        // (its geometry keeps every count below the prime), else over the 64-bit prime.
        const double mn = double(n) * double(m);
        path = mn <= 4.0e9 ? PA_PATH_DIRECT : PA_PATH_NTT31;
        TransformCfg probe;
        if (path == PA_PATH_NTT31 && ntt_plan(n, m, path, o, &probe) != PA_OK)
            path = PA_PATH_NTT64;
        if (path == PA_PATH_NTT64 && ntt_plan(n, m, path, o, &probe) != PA_OK)
            path = PA_PATH_DIRECT;
    }
    cfg->path = path;
    int rc = PA_OK;
    switch (path) {
        case PA_PATH_DIRECT:
            rc = direct_plan(n, m, &cfg->direct);
            cfg->ws_bytes = direct_workspace(cfg->direct);
            cfg->kernels = 2;  // key reversal (with output zeroing) and the direct kernel
            break;
        case PA_PATH_NTT64:
        case PA_PATH_NTT31:
            rc = ntt_plan(n, m, path, o, &cfg->tr);
            // Every standard tile pair is a tile record and several work items. A forced
            // geometry of tiny tiles on a long key (1e8 bits in 4096-bit tiles: 6e7 pairs),
            // or a key of 1e10 bits with transform-domain sums forbidden (2.3e6 pairs of
            // 2^22 points, 3e9 work items), would take minutes and tens of gigabytes of host
            // memory to lay out, so either is refused before any list is built.
            if (rc == PA_OK && cfg->tr.fd == 0 &&
                (double(cfg->tr.tiles_in) * double(cfg->tr.tiles_out) > double(kStdMaxPairs) ||
                 std_items(cfg->tr) > double(kStdMaxItems)))
                rc = PA_ERR_UNSUPPORTED;
            if (rc == PA_OK && (layout || (cfg->tr.fd == 1 && cfg->tr.seg_in)))
                rc = ntt_layout(n, m, path, &cfg->tr);
            cfg->ws_bytes = cfg->tr.lay.bytes;
            // output zeroing + the persistent launch (one per segment when segmented)
            cfg->kernels = 1 + static_cast<uint32_t>(std::max<size_t>(1, cfg->tr.segs.size()));
            break;
        case PA_PATH_FFT:
            rc = fft_plan(n, m, o, &cfg->tr);
            cfg->ws_bytes = fft_workspace(cfg->tr);
            cfg->kernels = 1 + static_cast<uint32_t>((cfg->tr.tiles_in * cfg->tr.tiles_out) >> 30);
            break;
        case PA_PATH_BLOCK_INT8:
            rc = block_plan(n, m, o, &cfg->blk);
            cfg->ws_bytes = block_workspace(cfg->blk);
            cfg->kernels = 2;  // key reversal (with output zeroing) and the contraction
            break;
        case PA_PATH_BLOCK_FP8:
            rc = block_tc_plan(n, m, o, &cfg->blk);
            cfg->ws_bytes = block_workspace(cfg->blk);
            cfg->kernels = 2;  // key reversal (with output zeroing) and the MMA kernel
            break;
    }
    return rc;
}

void fill_desc(const PlanCfg &cfg, pa_plan_desc *d) {
    memset(d, 0, sizeof(*d));
    d->n = cfg.n;
    d->m = cfg.m;
    d->path = cfg.path;
    d->workspace_bytes = cfg.ws_bytes + kHeaderBytes;
    d->kernels_per_call = cfg.kernels;
    if (cfg.path == PA_PATH_DIRECT) {
        d->tile_in = cfg.n;
        d->tile_out = cfg.m;
        d->tiles_in = d->tiles_out = 1;
    } else if (cfg.path == PA_PATH_BLOCK_FP8) {
        // tcgen05 kernel: contraction chunks of tile_in positions (one CTA each, FP32 sums
        // exact because tile_in <= 2^15), output tiles of 256 blocks of b rows
        d->block_b = cfg.blk.b;
        d->tile_in = cfg.blk.kc;
        d->tiles_in = cfg.blk.grid_x;
        d->tile_out = uint64_t(cfg.blk.b) * 256;
        d->tiles_out = cfg.blk.grid_y;
    } else if (cfg.path == PA_PATH_BLOCK_INT8) {
        d->block_b = cfg.blk.b;
        d->tile_in = cfg.n;
        d->tile_out = cfg.m;
        d->tiles_in = d->tiles_out = 1;
    } else {
        d->log2_transform = cfg.tr.log2n;
        d->tile_in = cfg.tr.L;
        d->tile_out = cfg.tr.M;
        d->tiles_in = cfg.tr.tiles_in;
        d->tiles_out = cfg.tr.tiles_out;
        d->fp64 = cfg.tr.fp64;
        d->rounding_bound = cfg.tr.bound;
        d->fd = cfg.tr.fd;
        d->windows = cfg.tr.windows;
        d->sum_groups = cfg.tr.fd == 1 && cfg.tr.kgroup
                            ? static_cast<uint32_t>(ceil_div(cfg.tr.tiles_in, cfg.tr.kgroup))
                            : (cfg.tr.fd ? 1u : 0u);
        d->outer_log2 = cfg.tr.outer_logT;
        d->outer_slice = cfg.tr.outer_slice;
        if (!cfg.tr.segs.empty()) {
            // every key segment has its own sums (one per kgroup key tiles of the segment)
            const uint64_t Sk = ceil_div(cfg.tr.tiles_in, cfg.tr.seg_in);
            d->sum_groups = static_cast<uint32_t>(Sk * ceil_div(cfg.tr.seg_in, cfg.tr.kgroup));
            d->seg_in = cfg.tr.seg_in;
            d->seg_out = cfg.tr.seg_out;
            d->segments = cfg.tr.segs.size();
        }
        if (cfg.path == PA_PATH_NTT31 || cfg.path == PA_PATH_NTT64)
            d->prime_bits = cfg.tr.field == kFieldF64   ? 64
                            : cfg.tr.field == kFieldF29 ? 29
                            : cfg.tr.field == kFieldF28 ? 28
                                                        : 31;
    }
}

}  // namespace pa

struct pa_plan_s {
    pa::PlanCfg cfg;
    int device = 0;
    void *mem = nullptr;  // header + workspace
    uint64_t *stage = nullptr;  // pa_hash_host staging: seed | key | out
    size_t stage_words = 0;
    cudaStream_t last_stream = nullptr;
    pa::Prof prof;
};

using namespace pa;

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int launch_plan(pa_plan_s *p, const uint64_t *seed, const uint64_t *key, uint64_t *out,
                cudaStream_t s) {
    DevHeader *hdr = static_cast<DevHeader *>(p->mem);
    void *ws = static_cast<char *>(p->mem) + kHeaderBytes;
    switch (p->cfg.path) {
        case PA_PATH_DIRECT: return direct_launch(p->cfg, ws, hdr, &p->prof, seed, key, out, s);
        case PA_PATH_NTT64:
        case PA_PATH_NTT31: return ntt_launch(p->cfg, ws, hdr, &p->prof, seed, key, out, s);
        case PA_PATH_FFT: return fft_launch(p->cfg, ws, hdr, &p->prof, seed, key, out, s);
        case PA_PATH_BLOCK_INT8:
        case PA_PATH_BLOCK_FP8: return block_launch(p->cfg, ws, hdr, &p->prof, seed, key, out, s);
    }
    return PA_ERR_INVALID;
}

}  // namespace

extern "C" {

int pa_plan_query(uint64_t n, uint64_t m, const pa_opts *opts, pa_plan_desc *out) {
    return guarded([&] {
        if (!out) return PA_ERR_INVALID;
        PlanCfg cfg;
        int rc = plan_resolve(n, m, opts, &cfg);
        if (rc != PA_OK) return rc;
        fill_desc(cfg, out);
        return PA_OK;
    });
}

int pa_seed_from_eq1(uint64_t n, const uint64_t *t_bits, uint64_t *seed_bits) {
    if (n == 0 || !t_bits || !seed_bits || n > kMaxBits) return PA_ERR_INVALID;
    const uint64_t len = 2 * n - 1, words = (len + 63) / 64;
    for (uint64_t w = 0; w < words; ++w) seed_bits[w] = 0;
    auto get = [t_bits](uint64_t i) { return (t_bits[i >> 6] >> (i & 63)) & 1u; };
    auto set = [seed_bits](uint64_t i) { seed_bits[i >> 6] |= uint64_t(1) << (i & 63); };
    for (uint64_t d = 0; d < n; ++d)  // on and below the diagonal
        if (get(d)) set(n - 1 + d);
    for (uint64_t e = 1; e < n; ++e)  // above it
        if (get(n - 1 + e)) set(n - 1 - e);
    return PA_OK;
}

int pa_plan_ex(uint64_t n, uint64_t m, const pa_opts *opts, pa_plan_t *out) {
    if (!out) return PA_ERR_INVALID;
    *out = nullptr;
    if (!sizes_valid(n, m)) return PA_ERR_INVALID;
    pa_plan_s *p = new (std::nothrow) pa_plan_s();
    if (!p) return PA_ERR_NOMEM;
    pa_opts tuned;
    if (!opts || opts->path == PA_PATH_AUTO) {
        // AUTO: the autotuner's measured-cost choice (calibrates once per device)
        const int trc = guarded([&] { return tuned_opts(n, m, &tuned); });
        if (trc != PA_OK) {
            delete p;
            return trc;
        }
        if (opts) tuned.device = opts->device;
        opts = &tuned;
    }
    int rc = guarded([&] { return plan_resolve(n, m, opts, &p->cfg); });
    if (rc != PA_OK) {
        delete p;
        return rc;
    }
    int prev = 0;
    cudaError_t e = cudaGetDevice(&prev);
    if (e != cudaSuccess) {
        delete p;
        return cuda_fail(e);
    }
    p->device = (opts && opts->device >= 0) ? opts->device : prev;
    if (p->device != prev && (e = cudaSetDevice(p->device)) != cudaSuccess) {
        delete p;
        return cuda_fail(e);
    }
    e = cudaMalloc(&p->mem, kHeaderBytes + p->cfg.ws_bytes);
    if (e == cudaSuccess) e = cudaMemset(p->mem, 0, kHeaderBytes);
    if (e == cudaSuccess && (p->cfg.path == PA_PATH_NTT31 || p->cfg.path == PA_PATH_NTT64)) {
        rc = guarded([&] { return ntt_init(p->cfg, static_cast<char *>(p->mem) + kHeaderBytes); });
        if (rc != PA_OK) {
            if (p->device != prev) cudaSetDevice(prev);
            cudaFree(p->mem);
            delete p;
            return rc;
        }
    }
    if (p->device != prev) cudaSetDevice(prev);
    if (e != cudaSuccess) {
        if (p->mem) cudaFree(p->mem);
        delete p;
        return cuda_fail(e);
    }
    *out = p;
    return PA_OK;
}

int pa_plan(uint64_t n, uint64_t m, pa_plan_t *out) { return pa_plan_ex(n, m, nullptr, out); }

int pa_plan_describe(pa_plan_t plan, pa_plan_desc *out) {
    if (!plan || !out) return PA_ERR_INVALID;
    fill_desc(plan->cfg, out);
    return PA_OK;
}

void pa_plan_destroy(pa_plan_t plan) {
    if (!plan) return;
    if (plan->last_stream) cudaStreamSynchronize(plan->last_stream);
    cudaFree(plan->mem);
    if (plan->stage) cudaFree(plan->stage);
    prof_free(&plan->prof);
    delete plan;
}

int pa_hash(pa_plan_t plan, const uint64_t *seed_bits, const uint64_t *key_bits,
            uint64_t *out_bits, void *stream) {
    return guarded([&] {
        if (!plan || !seed_bits || !key_bits || !out_bits) return PA_ERR_INVALID;
        if (!aligned16(seed_bits) || !aligned16(key_bits) || !aligned16(out_bits))
            return PA_ERR_ALIGN;
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        plan->last_stream = s;
        return launch_plan(plan, seed_bits, key_bits, out_bits, s);
    });
}

int pa_hash_host(pa_plan_t plan, const uint64_t *seed_host, const uint64_t *key_host,
                 uint64_t *out_host, void *stream) {
    if (!plan || !seed_host || !key_host || !out_host) return PA_ERR_INVALID;
    const uint64_t n = plan->cfg.n, m = plan->cfg.m;
    const size_t sw = round_up(ceil_div(n + m - 1, 64), 2), kw = round_up(ceil_div(n, 64), 2),
                 ow = round_up(ceil_div(m, 64), 2);
    if (!plan->stage) {
        cudaError_t e = cudaMalloc(&plan->stage, (sw + kw + ow) * 8);
        if (e != cudaSuccess) {
            plan->stage = nullptr;
            return cuda_fail(e);
        }
        plan->stage_words = sw + kw + ow;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t *dseed = plan->stage, *dkey = plan->stage + sw, *dout = plan->stage + sw + kw;
    PA_CUDA_TRY(cudaMemcpyAsync(dseed, seed_host, ceil_div(n + m - 1, 64) * 8,
                                cudaMemcpyHostToDevice, s));
    PA_CUDA_TRY(cudaMemcpyAsync(dkey, key_host, ceil_div(n, 64) * 8, cudaMemcpyHostToDevice, s));
    int rc = pa_hash(plan, dseed, dkey, dout, stream);
    if (rc != PA_OK) return rc;
    PA_CUDA_TRY(cudaMemcpyAsync(out_host, dout, ceil_div(m, 64) * 8, cudaMemcpyDeviceToHost, s));
    PA_CUDA_TRY(cudaStreamSynchronize(s));
    return PA_OK;
}

int pa_plan_status(pa_plan_t plan) {
    if (!plan) return PA_ERR_INVALID;
    PA_CUDA_TRY(cudaStreamSynchronize(plan->last_stream));
    DevHeader h;
    PA_CUDA_TRY(cudaMemcpy(&h, plan->mem, sizeof(h), cudaMemcpyDeviceToHost));
    if (h.status != 0) {
        int zero = 0;
        PA_CUDA_TRY(cudaMemcpy(plan->mem, &zero, sizeof(zero), cudaMemcpyHostToDevice));
    }
    return h.status;
}

int pa_last_residual(pa_plan_t plan, double *residual, double *bound) {
    if (!plan || !residual) return PA_ERR_INVALID;
    if (plan->last_stream) PA_CUDA_TRY(cudaStreamSynchronize(plan->last_stream));
    DevHeader h;
    PA_CUDA_TRY(cudaMemcpy(&h, plan->mem, sizeof(h), cudaMemcpyDeviceToHost));
    double r;
    memcpy(&r, &h.residual_bits, sizeof(r));
    *residual = r;
    if (bound) *bound = plan->cfg.tr.bound;
    unsigned long long zero = 0;
    PA_CUDA_TRY(cudaMemcpy(static_cast<char *>(plan->mem) + offsetof(DevHeader, residual_bits),
                           &zero, sizeof(zero), cudaMemcpyHostToDevice));
    return PA_OK;
}

int pa_plan_profile(pa_plan_t plan, int enable) {
    if (!plan) return PA_ERR_INVALID;
    return prof_enable(&plan->prof, enable);
}

int pa_plan_kernel_times(pa_plan_t plan, pa_kernel_time *out, int max, int *count) {
    if (!plan || max < 0) return PA_ERR_INVALID;
    return prof_collect(&plan->prof, out, max, count);
}

const char *pa_strerror(int status) {
    switch (status) {
        case PA_OK: return "success";
        case PA_ERR_INVALID: return "invalid argument (zero size, null pointer or bad option)";
        case PA_ERR_ALIGN: return "device bit buffer is not 16-byte aligned";
        case PA_ERR_NOMEM: return "out of memory";
        case PA_ERR_CUDA: return "CUDA runtime error";
        case PA_ERR_TIMEOUT: return "a bounded device-side wait timed out";
        case PA_ERR_UNSUPPORTED: return "sizes not supported by the requested path";
        case PA_ERR_PRECISION: return "no proven rounding bound below 1/2 for this FFT tile";
        case PA_ERR_TOO_LARGE: return "sizes exceed the fixed scratch of pa_hash_direct_static";
    }
    return "unknown status";
}

int pa_last_cuda_error(void) { return g_last_cuda_error; }

int pa_version(void) { return 100; }

}  // extern "C"
