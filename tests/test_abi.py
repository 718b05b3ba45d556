"""The C-ABI library loads and exports what include/pa.h declares (no GPU needed)."""
import os
import re

import pytest

import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "pa.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pa_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1805_02372_gb300 import build
    build.build()
    return binding.load()


def test_exports_every_declared_symbol(lib):
    names = header_functions()
    assert "pa_hash" in names and "pa_hash_batched" in names and "pa_plan" in names
    for name in names:
        assert hasattr(lib, name), f"{name} declared in pa.h but not exported"
        assert name in binding.SIGNATURES, f"{name} has no binding"


def test_strerror_and_version(lib):
    for code in range(0, -9, -1):
        assert pkg.pa_strerror(code) and pkg.pa_strerror(code) != "unknown status"
    assert pkg.pa_strerror(-99) == "unknown status"
    assert pkg.pa_version() >= 100


def test_plan_query_validates(lib):
    with pytest.raises(pkg.PAError) as e:
        pkg.pa_plan_query(0, 5)
    assert e.value.status == binding.PA_ERR_INVALID
    with pytest.raises(pkg.PAError):
        pkg.pa_plan_query(5, 0)
    with pytest.raises(pkg.PAError):
        pkg.pa_plan_query(5, 5, binding.make_opts(path=17))


@pytest.mark.parametrize("n,m", [(1, 1), (100_003, 25_000), (1_000_000, 500_000)])
def test_plan_query_direct(lib, n, m):
    d = pkg.pa_plan_query(n, m, binding.make_opts(path="direct"))
    assert d["path_name"] == "direct" and d["n"] == n and d["m"] == m
    assert d["workspace_bytes"] >= 4 * ((n + 31) // 32)


def test_fft_bound_properties(lib):
    b = pkg.pa_fft_rounding_bound
    # grows with the key tile, the output tile and the transform size; FP64 far smaller
    assert b(12, 512, 1024, False) < b(12, 1024, 1024, False) < b(12, 1024, 2048, False)
    assert b(11, 512, 512, False) < b(12, 512, 512, False)
    assert b(12, 2048, 2048, True) < 1e-8 < b(12, 32, 64, False)
    # the worst-case inverse term alone: alpha * L * sqrt(L + M) with alpha >= k * u
    assert b(12, 2048, 2048, False) > 12 * 2 ** -24 * 2048 * 4096 ** 0.5


@pytest.mark.parametrize("n,m", [(1, 1), (100_003, 25_000), (1_000_000, 500_000),
                                 (100_000_007, 10_000_000)])
def test_fft_planner_stays_under_half(lib, n, m):
    d = pkg.pa_plan_query(n, m, binding.make_opts(path="fft"))
    assert d["fp64"] == 0 and 0 < d["rounding_bound"] < 0.5
    assert d["tile_in"] + d["tile_out"] <= 1 << d["log2_transform"]
    assert d["rounding_bound"] == pkg.pa_fft_rounding_bound(d["log2_transform"], d["tile_in"],
                                                            d["tile_out"], False)


def test_fft_fp64_only_where_fp32_bound_fails(lib):
    # N = 2^12 with L = M = 2048: the FP32 bound exceeds 1/2, so FP64 butterflies.
    d = pkg.pa_plan_query(100_000, 50_000, binding.make_opts(path="fft", log2_transform=12,
                                                              tile_in=2048, tile_out=2048))
    assert d["fp64"] == 1 and d["rounding_bound"] < 1e-8
    d = pkg.pa_plan_query(100_000, 50_000, binding.make_opts(path="fft", log2_transform=12,
                                                              tile_in=1024, tile_out=2048))
    assert d["fp64"] == 0 and d["rounding_bound"] < 0.5


@pytest.mark.parametrize("n,m", [(1, 1), (100_003, 25_000), (1_000_000, 500_000),
                                 (100_000_007, 10_000_000), (3_000_000, 40_000)])
def test_plan_query_block_fp8(lib, n, m):
    # The tcgen05 block kernel sums at most one chunk of contraction positions per CTA in
    # FP32 (products 2^-12 each): chunks of at most 2^15 keep every partial sum exact. The
    # chunks cover the contraction n + 128 * 255 of every output tile of 256 x 128 outputs.
    d = pkg.pa_plan_query(n, m, binding.make_opts(path="block_fp8"))
    assert d["path_name"] == "block_fp8" and d["block_b"] == 128
    chunk, chunks, tiles = d["tile_in"], d["tiles_in"], d["tiles_out"]
    assert chunk % 128 == 0 and 1024 <= chunk <= 1 << 15
    assert chunks * chunk >= n + 128 * 255 > (chunks - 1) * chunk
    assert d["tile_out"] == 32768 and tiles == -(-m // 32768)
    assert d["kernels_per_call"] == 2
    with pytest.raises(pkg.PAError) as e:
        pkg.pa_plan_query(n, m, binding.make_opts(path="block_fp8", block_b=256))
    assert e.value.status == binding.PA_ERR_INVALID


@pytest.mark.parametrize("n,m", [(1_000_000_007, 100_000_000), (300_000_007, 30_000_000),
                                 (3_000_000_000, 300_000_000)])
def test_plan_query_paper_scale(lib, n, m):
    # Paper-scale blocks (Fig. 3 reaches 1e10 bits): the exact transform over the 29-bit
    # prime at any length, with transform-domain accumulation so only (key + window +
    # output) spectra of N <= 2^23 elements are held. A sum over g key tiles counts at
    # most g L products per coefficient, so each output tile takes ceil(Q / g) sums with
    # g = (p - 1) // L, and their bits are XOR-merged.
    p29 = 7 * 2 ** 26 + 1
    d = pkg.pa_plan_query(n, m)
    assert d["path_name"] == "ntt31" and d["prime_bits"] == 29
    k, L, Q, P = d["log2_transform"], d["tile_in"], d["tiles_in"], d["tiles_out"]
    assert k <= 23 and d["fd"] == 1
    g = (p29 - 1) // L
    assert d["sum_groups"] == -(-Q // g) and (n <= p29 - 1 or d["sum_groups"] >= 2)
    # resident spectra: key tiles + distinct windows + one output per sum
    assert d["workspace_bytes"] >= 4 * (Q + d["windows"] + d["sum_groups"] * P) << k
    assert d["workspace_bytes"] < 96 * 2 ** 30


@pytest.mark.parametrize("n", [1, 2, 3, 31, 32, 33, 64, 65, 1000, 4097])
def test_seed_from_eq1_matches_oracle(lib, n):
    # The library's Eq. 1 helper against the oracle's (itself pinned to a literal Eq. 1
    # matrix in test_oracle.py); the two are written independently.
    import numpy as np
    import oracle
    rng = np.random.default_rng(n)
    t = rng.integers(0, 2, 2 * n - 1, dtype=np.uint8)
    words = (2 * n - 1 + 63) // 64
    tw = np.zeros(words, dtype=np.uint64)
    for i in np.flatnonzero(t):
        tw[i >> 6] |= np.uint64(1) << np.uint64(i & 63)
    tw[-1] |= ~np.uint64(0) << np.uint64((2 * n - 1) % 64) if (2 * n - 1) % 64 else np.uint64(0)
    got = binding.pa_seed_from_eq1(n, tw)
    assert np.array_equal(oracle.unpack(got, 2 * n - 1), oracle.seed_from_eq1(t))
    if (2 * n - 1) % 64:
        assert int(got[-1]) >> ((2 * n - 1) % 64) == 0
    with pytest.raises(pkg.PAError):
        binding.pa_seed_from_eq1(0, tw)


NOMEM_DRIVER = r'''
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <sys/resource.h>
#include "pa.h"
/* the process's current address-space size in bytes (VmSize of /proc/self/status) */
static long vm_bytes(void) {
    FILE *f = fopen("/proc/self/status", "r");
    char line[256];
    long kb = -1;
    while (f && fgets(line, sizeof(line), f))
        if (strncmp(line, "VmSize:", 7) == 0) kb = atol(line + 7);
    if (f) fclose(f);
    return kb * 1024;
}
int main(int argc, char **argv) {
    pa_plan_desc d;
    pa_opts o;
    memset(&o, 0, sizeof(o));
    o.device = -1;
    o.path = PA_PATH_NTT31;
    o.fd_mode = 1;
    if (argc > 1) {  /* leave this process 96 MiB above what it holds now */
        const long vm = vm_bytes();
        if (vm <= 0) return 2;
        struct rlimit r = {(rlim_t)vm + (96l << 20), (rlim_t)vm + (96l << 20)};
        if (setrlimit(RLIMIT_AS, &r) != 0) return 3;
    }
    const int big = pa_plan_query(1000000007ull, 100000000ull, &o, &d);
    const int small = pa_plan_query(100003, 25000, NULL, &d);
    printf("%d %d\n", big, small);
    return 0;
}
'''


def test_host_allocation_failure_is_a_status(lib, tmp_path):
    # A 1e9-bit key with transform-domain sums forbidden lays out 2.3e4 standard tile pairs,
    # about 3e7 work items (230 MB of list). With the process's address space capped 96 MiB
    # above its size, the list cannot grow: the C interface must return PA_ERR_NOMEM
    # (std::bad_alloc caught at the boundary), not terminate, and stay usable afterwards.
    import shutil
    import subprocess
    from paper_1805_02372_gb300 import build
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src, exe = tmp_path / "nomem.c", tmp_path / "nomem"
    src.write_text(NOMEM_DRIVER)
    r = subprocess.run(["gcc", "-O1", "-I", os.path.join(ROOT, "include"), str(src), build.LIB,
                        "-Wl,-rpath," + os.path.dirname(build.LIB), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    free = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert free.returncode == 0 and free.stdout.split() == ["0", "0"], free.stdout + free.stderr
    capped = subprocess.run([str(exe), "cap"], capture_output=True, text=True, timeout=300)
    assert capped.returncode == 0, capped.stdout + capped.stderr
    assert capped.stdout.split() == [str(binding.PA_ERR_NOMEM), "0"], capped.stdout


INVALID_DRIVER = r'''
#include <stdio.h>
#include <string.h>
#include "pa.h"
static int fails = 0;
#define EXPECT(call, want)                                                        \
    do {                                                                          \
        const int got_ = (call);                                                  \
        if (got_ != (want)) {                                                     \
            printf("FAIL %s -> %d, expected %d\n", #call, got_, (int)(want));     \
            ++fails;                                                              \
        }                                                                         \
    } while (0)
int main(void) {
    static uint64_t buf[8] __attribute__((aligned(16)));
    uint64_t *odd = (uint64_t *)((char *)buf + 8);
    pa_plan_desc d;
    pa_plan_t plan = (pa_plan_t)0;
    pa_batch_t batch = (pa_batch_t)0;
    pa_server_t server = (pa_server_t)0;
    pa_block blk = {1000, 100, buf, buf, buf};
    pa_report rep;
    pa_completion done[4];
    pa_server_stats st;
    pa_kernel_time kt[4];
    size_t count = 0;
    int n = 0;
    double r = 0, b = 0;
    /* plans */
    EXPECT(pa_plan(0, 5, &plan), PA_ERR_INVALID);
    EXPECT(pa_plan(5, 5, NULL), PA_ERR_INVALID);
    EXPECT(pa_plan_ex(5, 0, NULL, &plan), PA_ERR_INVALID);
    EXPECT(pa_plan_ex((uint64_t)1 << 41, 5, NULL, &plan), PA_ERR_INVALID);
    EXPECT(pa_plan_query(5, 5, NULL, NULL), PA_ERR_INVALID);
    EXPECT(pa_plan_describe(NULL, &d), PA_ERR_INVALID);
    EXPECT(pa_hash(NULL, buf, buf, buf, NULL), PA_ERR_INVALID);
    EXPECT(pa_hash_host(NULL, buf, buf, buf, NULL), PA_ERR_INVALID);
    EXPECT(pa_last_residual(NULL, &r, &b), PA_ERR_INVALID);
    EXPECT(pa_plan_status(NULL), PA_ERR_INVALID);
    EXPECT(pa_plan_profile(NULL, 1), PA_ERR_INVALID);
    EXPECT(pa_plan_kernel_times(NULL, kt, 4, &n), PA_ERR_INVALID);
    pa_plan_destroy(NULL);
    /* the no-allocation entry point: sizes and alignment first */
    EXPECT(pa_hash_direct_static(0, 5, buf, buf, buf, NULL), PA_ERR_INVALID);
    EXPECT(pa_hash_direct_static(5, 5, NULL, buf, buf, NULL), PA_ERR_INVALID);
    EXPECT(pa_hash_direct_static(5, 5, odd, buf, buf, NULL), PA_ERR_ALIGN);
    EXPECT(pa_hash_direct_static((uint64_t)1 << 26, 5, buf, buf, buf, NULL), PA_ERR_TOO_LARGE);
    /* batches */
    EXPECT(pa_batch_plan(NULL, 1, NULL, &batch), PA_ERR_INVALID);
    EXPECT(pa_batch_plan(&blk, 0, NULL, &batch), PA_ERR_INVALID);
    EXPECT(pa_batch_plan(&blk, 1, NULL, NULL), PA_ERR_INVALID);
    blk.n = (uint64_t)1 << 41;  /* refused before the autotuner calibrates */
    EXPECT(pa_batch_plan(&blk, 1, NULL, &batch), PA_ERR_INVALID);
    blk.n = 1000;
    EXPECT(pa_batch_run(NULL, &blk, 1, NULL, &rep), PA_ERR_INVALID);
    EXPECT(pa_batch_run_host(NULL, &blk, 1, NULL, &rep), PA_ERR_INVALID);
    EXPECT(pa_batch_run_host_async(NULL, &blk, 1, NULL), PA_ERR_INVALID);
    EXPECT(pa_batch_get_report(NULL, NULL, &rep), PA_ERR_INVALID);
    EXPECT(pa_batch_describe(NULL, &d, 1), PA_ERR_INVALID);
    EXPECT(pa_batch_profile(NULL, 1), PA_ERR_INVALID);
    EXPECT(pa_batch_kernel_times(NULL, kt, 4, &n), PA_ERR_INVALID);
    EXPECT(pa_hash_batched(NULL, 1, NULL, &rep), PA_ERR_INVALID);
    EXPECT(pa_hash_batched(&blk, 0, NULL, &rep), PA_ERR_INVALID);
    pa_batch_destroy(NULL);
    /* server */
    EXPECT(pa_server_create(NULL, NULL), PA_ERR_INVALID);
    EXPECT(pa_server_submit(NULL, &blk, 1), PA_ERR_INVALID);
    EXPECT(pa_server_poll(NULL, done, 4, &count), PA_ERR_INVALID);
    EXPECT(pa_server_pending(NULL, NULL, NULL), PA_ERR_INVALID);
    EXPECT(pa_server_get_stats(NULL, &st), PA_ERR_INVALID);
    pa_server_destroy(NULL);
    /* host helpers and probes */
    EXPECT(pa_seed_from_eq1(0, buf, buf), PA_ERR_INVALID);
    EXPECT(pa_seed_from_eq1(5, NULL, buf), PA_ERR_INVALID);
    EXPECT(pa_fft_rounding_bound(0, 64, 64, 0, &r), PA_ERR_INVALID);
    EXPECT(pa_fft_rounding_bound(12, 64, 64, 0, NULL), PA_ERR_INVALID);
    EXPECT(pa_probe_peak(-1, &r, &b), PA_ERR_INVALID);
    EXPECT(pa_probe_peak(0, NULL, &b), PA_ERR_INVALID);
    EXPECT(pa_selftest(0, &n), PA_ERR_INVALID);
    EXPECT(pa_selftest(1, NULL), PA_ERR_INVALID);
    /* none of the above reached the CUDA runtime */
    EXPECT(pa_last_cuda_error(), 0);
    printf("done %d\n", fails);
    return fails != 0;
}
'''


def test_invalid_arguments_refused_before_any_cuda_call(lib, tmp_path):
    # Every entry point checks its handle, pointers, sizes and alignment before it touches
    # the CUDA runtime: on this machine (no GPU) each call returns its documented status,
    # and the last CUDA error stays 0 (a CUDA call would have failed here and set it).
    import shutil
    import subprocess
    from paper_1805_02372_gb300 import build
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    src, exe = tmp_path / "invalid.c", tmp_path / "invalid"
    src.write_text(INVALID_DRIVER)
    r = subprocess.run(["gcc", "-O1", "-Wall", "-I", os.path.join(ROOT, "include"), str(src),
                        build.LIB, "-Wl,-rpath," + os.path.dirname(build.LIB), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert run.returncode == 0 and run.stdout.strip().endswith("done 0"), run.stdout + run.stderr


@pytest.mark.parametrize("compiler,std", [("gcc", "-std=c99"), ("g++", "-std=c++11")])
def test_header_compiles_strictly(tmp_path, compiler, std):
    # include/pa.h is a C interface: plain C99 and C++11 with every warning an error
    import shutil
    import subprocess
    if not shutil.which(compiler):
        pytest.skip(f"{compiler} not available")
    src = tmp_path / ("h.c" if compiler == "gcc" else "h.cpp")
    src.write_text('#include "pa.h"\n'
                   "int main(void) { pa_plan_desc d; pa_opts o; pa_block b; pa_report r;\n"
                   "  (void)d; (void)o; (void)b; (void)r; return pa_version() > 0 ? 0 : 1; }\n")
    r = subprocess.run([compiler, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-I",
                        os.path.join(ROOT, "include"), "-c", str(src), "-o", os.devnull],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
