#include "internal.h"
namespace pa {
int fft_plan(uint64_t, uint64_t, const pa_opts *, TransformCfg *) { return PA_ERR_UNSUPPORTED; }
size_t fft_workspace(const TransformCfg &) { return 0; }
int fft_launch(const PlanCfg &, void *, DevHeader *, Prof *, const uint64_t *, const uint64_t *, uint64_t *, cudaStream_t) { return PA_ERR_UNSUPPORTED; }
}
