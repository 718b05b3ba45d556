// Serving: continuous batching of PA requests arriving from reconciliation by device
// memory (Sec. 3: the corrected keys are already on the GPU, so no copy is needed).
//
// A server owns S stream slots and a device-memory budget. Submitted requests wait in a
// FIFO; whenever a slot is free, the requests waiting at that moment (up to a cap, and
// while their batch workspace fits the budget left by the waves in flight) are planned
// as one batch (one persistent launch for the transform blocks) and launched on that
// slot's stream. Waves on different slots overlap on the device, so requests arriving
// while others run are admitted as slots and memory free up. Completion is an event
// per wave; poll returns finished requests with their tags.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include "guard.h"
#include "internal.h"

namespace {

struct Wave {
    pa_batch_t batch = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<uint64_t> tags;
    size_t bytes = 0;
    int status = PA_OK;
};

}  // namespace

struct pa_server_s {
    int device = 0;
    pa_server_opts opts;
    std::mutex mu;
    std::deque<std::pair<pa_block, uint64_t>> queue;
    std::vector<cudaStream_t> streams;
    std::vector<Wave> slots;  // one (possibly empty) wave per slot
    size_t bytes_in_flight = 0;
    uint64_t waves_launched = 0, requests_done = 0;
    double plan_s_total = 0, plan_s_max = 0;  // host time of launch_wave per launched wave
    uint64_t held_back = 0;                   // waves held back by the memory budget
};

using namespace pa;

namespace {

bool slot_busy(const Wave &w) { return w.batch != nullptr; }

int launch_wave_impl(pa_server_s *s, size_t i);

// Launch one wave on slot i from the head of the queue. Called with the lock held. Records
// the host time it took (planning, workspace, upload, launch) for pa_server_get_stats.
int launch_wave(pa_server_s *s, size_t i) {
    const auto t0 = std::chrono::steady_clock::now();
    const uint64_t before = s->waves_launched;
    const int rc = launch_wave_impl(s, i);
    const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (s->waves_launched != before) {
        s->plan_s_total += dt;
        if (dt > s->plan_s_max) s->plan_s_max = dt;
    }
    return rc;
}

int launch_wave_impl(pa_server_s *s, size_t i) {
    // The wave takes the requests at the head of the queue; they leave the queue only once
    // the wave is launched, so a failed plan or a held-back wave leaves them waiting in order.
    const size_t cap = s->opts.max_blocks_per_wave ? s->opts.max_blocks_per_wave : 64;
    const size_t k = std::min(s->queue.size(), cap);
    if (k == 0) return PA_OK;
    std::vector<pa_block> blocks;
    std::vector<uint64_t> tags;
    blocks.reserve(k);
    tags.reserve(k);
    for (size_t j = 0; j < k; ++j) {
        blocks.push_back(s->queue[j].first);
        tags.push_back(s->queue[j].second);
    }
    Wave w;
    pa_batch_s *b = nullptr;
    int rc = batch_plan_impl(blocks.data(), blocks.size(), nullptr, s->streams[i], true, &b);
    if (rc != PA_OK) return rc;
    w.batch = b;
    w.bytes = batch_bytes(b);
    // memory admission: a wave that does not fit next to the waves in flight waits for
    // them (its plan is released in stream order; nothing ran yet)
    if (s->opts.memory_budget_bytes && s->bytes_in_flight > 0 &&
        s->bytes_in_flight + w.bytes > s->opts.memory_budget_bytes) {
        batch_destroy_impl(b);
        ++s->held_back;
        return PA_OK;
    }
    cudaError_t e = cudaEventCreateWithFlags(&w.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        batch_destroy_impl(w.batch);
        return cuda_fail(e);
    }
    rc = pa_batch_run(w.batch, blocks.data(), blocks.size(), s->streams[i], nullptr);
    if (rc == PA_OK) {
        e = cudaEventRecord(w.done, s->streams[i]);
        if (e != cudaSuccess) rc = cuda_fail(e);
    }
    // launched (or failed on launch): the requests leave the queue and complete with the
    // wave's status; nothing below allocates
    for (size_t j = 0; j < k; ++j) s->queue.pop_front();
    w.status = rc;
    w.tags = std::move(tags);
    s->bytes_in_flight += w.bytes;
    s->slots[i] = std::move(w);
    ++s->waves_launched;
    return PA_OK;
}

}  // namespace

extern "C" {

int pa_server_create(const pa_server_opts *opts, pa_server_t *out) {
    if (!out) return PA_ERR_INVALID;
    *out = nullptr;
    pa_server_s *s = new (std::nothrow) pa_server_s();
    if (!s) return PA_ERR_NOMEM;
    memset(&s->opts, 0, sizeof(s->opts));
    if (opts) s->opts = *opts;
    if (s->opts.slots == 0) s->opts.slots = 2;
    if (s->opts.slots > 64) s->opts.slots = 64;
    // the containers take their final sizes before any CUDA object exists
    const int grc = guarded([&] {
        s->streams.reserve(s->opts.slots);
        s->slots.resize(s->opts.slots);
        return PA_OK;
    });
    if (grc != PA_OK) {
        delete s;
        return grc;
    }
    cudaError_t e = cudaGetDevice(&s->device);
    for (uint32_t i = 0; e == cudaSuccess && i < s->opts.slots; ++i) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) s->streams.push_back(st);
    }
    if (e != cudaSuccess) {
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        delete s;
        return cuda_fail(e);
    }
    // keep freed wave memory in the device's stream-ordered pool for the next waves
    // (a property of this process's pool only)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
        uint64_t keep = ~uint64_t(0);
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    // calibrate the autotuner now, not while the first wave waits
    pa_opts warm;
    const int trc = guarded([&] { return tuned_opts(1 << 20, 1 << 16, &warm); });
    if (trc != PA_OK) {
        for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
        delete s;
        return trc;
    }
    *out = s;
    return PA_OK;
}

int pa_server_submit(pa_server_t s, const pa_block *req, uint64_t tag) {
    return guarded([&] {
        // a request no plan can take is refused here, not left to block the queue
        if (!s || !req || !sizes_valid(req->n, req->m) || !req->seed_bits || !req->key_bits ||
            !req->out_bits)
            return PA_ERR_INVALID;
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.push_back({*req, tag});
        return PA_OK;
    });
}

int pa_server_poll(pa_server_t s, pa_completion *done, size_t max, size_t *count) {
    return guarded([&] {
        if (!s || (!done && max) || !count) return PA_ERR_INVALID;
        std::lock_guard<std::mutex> lk(s->mu);
        *count = 0;
        // retire finished waves
        for (size_t i = 0; i < s->slots.size(); ++i) {
            Wave &w = s->slots[i];
            if (!slot_busy(w)) continue;
            if (w.tags.size() > max - *count) continue;  // no room to report this wave yet
            const cudaError_t q = cudaEventQuery(w.done);
            if (q == cudaErrorNotReady) continue;
            int st = w.status;
            if (q != cudaSuccess) st = cuda_fail(q);
            for (uint64_t t : w.tags) {
                done[*count].tag = t;
                done[*count].status = st;
                ++*count;
            }
            s->requests_done += w.tags.size();
            cudaEventDestroy(w.done);
            batch_destroy_impl(w.batch);
            s->bytes_in_flight -= w.bytes;
            w = Wave();
        }
        // admit: every free slot takes the requests waiting now
        for (size_t i = 0; i < s->slots.size() && !s->queue.empty(); ++i) {
            if (slot_busy(s->slots[i])) continue;
            int rc = launch_wave(s, i);
            if (rc != PA_OK) return rc;
            if (!slot_busy(s->slots[i])) break;  // held back by the memory budget
        }
        return PA_OK;
    });
}

int pa_server_pending(pa_server_t s, uint64_t *queued, uint64_t *in_flight) {
    if (!s) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = s->queue.size();
    uint64_t f = 0;
    for (const Wave &w : s->slots) f += w.tags.size();
    if (in_flight) *in_flight = f;
    return PA_OK;
}

int pa_server_get_stats(pa_server_t s, pa_server_stats *out) {
    if (!s || !out) return PA_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    memset(out, 0, sizeof(*out));
    out->waves = s->waves_launched;
    out->requests_done = s->requests_done;
    out->plan_s_total = s->plan_s_total;
    out->plan_s_max = s->plan_s_max;
    out->waves_held_back = s->held_back;
    return PA_OK;
}

void pa_server_destroy(pa_server_t s) {
    if (!s) return;
    for (cudaStream_t st : s->streams) cudaStreamSynchronize(st);
    for (Wave &w : s->slots) {
        if (w.done) cudaEventDestroy(w.done);
        if (w.batch) batch_destroy_impl(w.batch);
    }
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
