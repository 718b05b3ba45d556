#include "internal.h"
namespace pa {
int ntt_plan(uint64_t, uint64_t, int, const pa_opts *, TransformCfg *) { return PA_ERR_UNSUPPORTED; }
size_t ntt_workspace(int, const TransformCfg &) { return 0; }
int ntt_launch(const PlanCfg &, void *, DevHeader *, Prof *, const uint64_t *, const uint64_t *, uint64_t *, cudaStream_t) { return PA_ERR_UNSUPPORTED; }
}
