// Persistent NTT launch over the prime field F28 (see ntt_kernel.cuh); one field per
// translation unit so the instantiations compile in parallel.
#include "ntt_kernel.cuh"

namespace pa {

int ntt_launch_f28(PA_NTT_LAUNCH_ARGS) {
    return launch_field<F28>(lay, ws, blks, one, status, prof, s);
}

}  // namespace pa
