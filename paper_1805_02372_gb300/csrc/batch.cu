#include "internal.h"
extern "C" {
int pa_batch_plan(const pa_block *, size_t, const pa_opts *, pa_batch_t *out) { if (out) *out = nullptr; return PA_ERR_UNSUPPORTED; }
int pa_batch_run(pa_batch_t, const pa_block *, size_t, void *, pa_report *) { return PA_ERR_UNSUPPORTED; }
void pa_batch_destroy(pa_batch_t) {}
int pa_batch_profile(pa_batch_t, int) { return PA_ERR_UNSUPPORTED; }
int pa_batch_kernel_times(pa_batch_t, pa_kernel_time *, int, int *) { return PA_ERR_UNSUPPORTED; }
int pa_hash_batched(const pa_block *, size_t, void *, pa_report *) { return PA_ERR_UNSUPPORTED; }
}
