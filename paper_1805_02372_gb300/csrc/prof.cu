// Per-kernel CUDA-event timing: an event pair around each launch while enabled.
#include <stdlib.h>
#include <string.h>

#include "internal.h"

namespace pa {

static const char *kNames[K_NUM_KERNELS] = {"reverse_key", "direct",           "fft_tile",
                                             "block_mma",   "batch_persistent", "memset",
                                             "block_tc"};

const char *kernel_name(int kid) { return (kid >= 0 && kid < K_NUM_KERNELS) ? kNames[kid] : "?"; }

static bool grow(Prof *p) {
    size_t cap = p->cap ? p->cap * 2 : 256;
    ProfRec *r = static_cast<ProfRec *>(realloc(p->recs, cap * sizeof(ProfRec)));
    if (!r) return false;
    for (size_t i = p->cap; i < cap; ++i) {
        r[i].kid = -1;
        if (cudaEventCreate(&r[i].a) != cudaSuccess || cudaEventCreate(&r[i].b) != cudaSuccess) {
            p->recs = r;
            p->cap = i;
            return false;
        }
    }
    p->recs = r;
    p->cap = cap;
    return true;
}

void prof_begin(Prof *p, int kid, cudaStream_t s) {
    if (!p || !p->on) return;
    if (p->used == p->cap && !grow(p)) return;
    p->recs[p->used].kid = kid;
    cudaEventRecord(p->recs[p->used].a, s);
    p->open_kid = kid;
}

void prof_end(Prof *p, cudaStream_t s) {
    if (!p || !p->on || p->open_kid < 0) return;
    cudaEventRecord(p->recs[p->used].b, s);
    ++p->used;
    p->open_kid = -1;
}

int prof_enable(Prof *p, int enable) {
    p->on = enable != 0;
    if (enable) p->used = 0;
    p->open_kid = -1;
    return PA_OK;
}

int prof_collect(Prof *p, pa_kernel_time *out, int max, int *count) {
    double tot[K_NUM_KERNELS] = {0};
    uint32_t cnt[K_NUM_KERNELS] = {0};
    for (size_t i = 0; i < p->used; ++i) {
        PA_CUDA_TRY(cudaEventSynchronize(p->recs[i].b));
        float ms = 0.f;
        PA_CUDA_TRY(cudaEventElapsedTime(&ms, p->recs[i].a, p->recs[i].b));
        tot[p->recs[i].kid] += ms;
        cnt[p->recs[i].kid] += 1;
    }
    int k = 0;
    for (int kid = 0; kid < K_NUM_KERNELS; ++kid) {
        if (!cnt[kid]) continue;
        if (k < max && out) {
            memset(&out[k], 0, sizeof(out[k]));
            strncpy(out[k].name, kNames[kid], sizeof(out[k].name) - 1);
            out[k].launches = cnt[kid];
            out[k].total_ms = tot[kid];
        }
        ++k;
    }
    if (count) *count = k < max ? k : max;
    return PA_OK;
}

void prof_free(Prof *p) {
    for (size_t i = 0; i < p->cap; ++i) {
        cudaEventDestroy(p->recs[i].a);
        cudaEventDestroy(p->recs[i].b);
    }
    free(p->recs);
    p->recs = nullptr;
    p->cap = p->used = 0;
}

}  // namespace pa
