"""GB300 (sm_103a) Toeplitz hash for length-compatible privacy amplification.

The hash y = T x mod 2 with T[i][j] = s[n-1+i-j] (arXiv 1805.02372, Sec. 2-3) runs
in the CUDA library ``_lib/libpa.so`` behind the C ABI of ``include/pa.h``;
``binding`` marshals arguments to it and ``inputs`` draws seeded synthetic bits.
Importing the package does not load the library; the first call does, and fails
loudly if it has not been built.
"""
from . import inputs, serve  # noqa: F401
from .binding import (BlockList, Plan, PAError, pa_batch_describe, pa_batch_destroy, pa_batch_run_host, pa_batch_plan, pa_batch_run,  # noqa: F401
                      pa_batch_kernel_times, pa_batch_profile, pa_batch_run_host_async, pa_batch_get_report,
                      pa_fft_rounding_bound, pa_hash, pa_hash_batched, pa_plan_kernel_times, pa_plan_profile, pa_hash_host, pa_last_residual, pa_plan,
                      pa_plan_describe, pa_plan_destroy, pa_plan_ex, pa_plan_query,
                      pa_plan_status, pa_server_create, pa_server_destroy, pa_server_pending,
                      pa_server_poll, pa_server_submit, pa_strerror, pa_version, make_opts)
