#include "internal.h"
namespace pa {
int block_plan(uint64_t, uint64_t, const pa_opts *, BlockCfg *) { return PA_ERR_UNSUPPORTED; }
size_t block_workspace(const BlockCfg &) { return 0; }
int block_launch(const PlanCfg &, void *, DevHeader *, Prof *, const uint64_t *, const uint64_t *, uint64_t *, cudaStream_t) { return PA_ERR_UNSUPPORTED; }
}
