// Persistent NTT launch over the prime field F31 (see ntt_kernel.cuh); one field per
// translation unit so the instantiations compile in parallel.
#include "ntt_kernel.cuh"

namespace pa {

int ntt_launch_f31(PA_NTT_LAUNCH_ARGS) {
    return launch_field<F31>(lay, ws, blks, one, status, prof, s);
}

}  // namespace pa
