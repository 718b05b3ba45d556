"""Host code under AddressSanitizer, UndefinedBehaviorSanitizer and ThreadSanitizer (no GPU).

Three instrumented programs are built and run here:

* the oracle (``oracle/pa_oracle.c``) with a driver that hands it buffers of exactly the
  sizes its interface states (a read or write one word past an end is reported), over
  ragged shapes from one bit up, with 1 and 4 threads; the test program also checks that the
  threaded hash, the packed row evaluator and the bit-by-bit evaluator of the definition
  (Sec. 2.1, Eq. 1) agree, and that invalid arguments are refused;
* the same oracle and driver under ThreadSanitizer (the threads write disjoint, 64-row
  aligned ranges of the output words; a race between them would be reported);
* the CUDA library's host code (planner, work-list builder, descriptor filling): every
  ``csrc/*.cu`` compiled with the instrumentation on its host side (device code as PTX
  only, never run), driven through the host-only entry points: ``pa_plan_query`` over
  shapes from one bit to 1e10 bits and at the interface's 2^40-bit limit, every path and
  every option family, including refused and invalid ones, ``pa_seed_from_eq1`` on
  exact-size buffers and ``pa_fft_rounding_bound``.

A finding aborts the program with its report and the test fails with it. One test plants
an off-by-one read in a copy of the oracle and checks the instrumented build reports it,
so a harness that could not see such a mistake fails too.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_SRC = os.path.join(ROOT, "oracle", "pa_oracle.c")
CSRC = os.path.join(ROOT, "paper_1805_02372_gb300", "csrc")
INCLUDE = os.path.join(ROOT, "include")
SAN_ENV = dict(os.environ, ASAN_OPTIONS="protect_shadow_gap=0:detect_leaks=0:abort_on_error=0",
               UBSAN_OPTIONS="print_stacktrace=1:halt_on_error=1",
               TSAN_OPTIONS="halt_on_error=1")

ORACLE_DRIVER = r'''
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int oracle_hash(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key,
                uint64_t *out, int nthreads);
int oracle_rows(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key,
                const uint64_t *rows, uint64_t count, uint8_t *bits, int nthreads);
int oracle_rows_bitloop(uint64_t n, uint64_t m, const uint64_t *seed, const uint64_t *key,
                        const uint64_t *rows, uint64_t count, uint8_t *bits);

static uint64_t state = 0x9E3779B97F4A7C15ull;
static uint64_t next_word(void) {  /* xorshift64 */
    state ^= state << 13;
    state ^= state >> 7;
    state ^= state << 17;
    return state;
}
/* exactly ceil(bits/64) words, every bit random (bits past the string's end too) */
static uint64_t *random_words(uint64_t bits) {
    const uint64_t w = (bits + 63) / 64;
    uint64_t *p = (uint64_t *)malloc(w * sizeof(uint64_t));
    for (uint64_t i = 0; i < w; ++i) p[i] = next_word();
    return p;
}
#define CHECK(c) do { if (!(c)) { printf("FAIL line %d n=%llu m=%llu\n", __LINE__, \
    (unsigned long long)n, (unsigned long long)m); return 1; } } while (0)

int main(void) {
    static const uint64_t shapes[][2] = {
        {1, 1}, {1, 64}, {64, 1}, {63, 65}, {65, 63}, {127, 129}, {1000, 1}, {1, 1000},
        {4097, 4095}, {70001, 3333}, {200003, 65}, {64, 64}, {128, 192}};
    const int ns = (int)(sizeof(shapes) / sizeof(shapes[0]));
    for (int s = 0; s < ns; ++s) {
        const uint64_t n = shapes[s][0], m = shapes[s][1], ow = (m + 63) / 64;
        uint64_t *seed = random_words(n + m - 1), *key = random_words(n);
        uint64_t *out1 = (uint64_t *)malloc(ow * 8), *out4 = (uint64_t *)malloc(ow * 8);
        CHECK(oracle_hash(n, m, seed, key, out1, 1) == 0);
        CHECK(oracle_hash(n, m, seed, key, out4, 4) == 0);
        CHECK(memcmp(out1, out4, ow * 8) == 0);
        if (m & 63) CHECK((out1[ow - 1] >> (m & 63)) == 0);
        const uint64_t count = m < 97 ? m : 97;
        uint64_t *rows = (uint64_t *)malloc(count * 8);
        for (uint64_t t = 0; t < count; ++t) rows[t] = (t * 7919u) % m;
        rows[count - 1] = m - 1;
        uint8_t *b4 = (uint8_t *)malloc(count), *bb = (uint8_t *)malloc(count);
        CHECK(oracle_rows(n, m, seed, key, rows, count, b4, 4) == 0);
        CHECK(oracle_rows_bitloop(n, m, seed, key, rows, count, bb) == 0);
        for (uint64_t t = 0; t < count; ++t) {
            CHECK(b4[t] == bb[t]);
            CHECK(b4[t] == ((out1[rows[t] >> 6] >> (rows[t] & 63)) & 1u));
        }
        /* invalid arguments are refused without touching memory */
        CHECK(oracle_hash(0, m, seed, key, out1, 1) != 0);
        CHECK(oracle_hash(n, m, seed, key, NULL, 1) != 0);
        rows[0] = m;
        CHECK(oracle_rows(n, m, seed, key, rows, count, b4, 2) != 0);
        CHECK(oracle_rows_bitloop(n, m, seed, key, rows, count, bb) != 0);
        CHECK(oracle_rows(n, m, seed, key, NULL, count, b4, 2) != 0);
        CHECK(oracle_rows_bitloop(n, m, seed, key, NULL, count, bb) != 0);
        free(seed); free(key); free(out1); free(out4); free(rows); free(b4); free(bb);
    }
    printf("ok %d shapes\n", ns);
    return 0;
}
'''

PLANNER_DRIVER = r'''
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include "pa.h"

static int variant(pa_opts *o, int v) {
    switch (v) {
        case 1: o->ntt_prime = 28; break;
        case 2: o->ntt_prime = 31; break;
        case 3: o->fd_mode = 1; break;
        case 4: o->fd_mode = 2; o->fd_group = 3; break;
        case 5: o->outer_mode = 2; break;
        case 6: o->outer_mode = 1; o->seg_in = 3; o->seg_out = 2; break;
        case 7: o->log2_transform = 13; o->tile_in = 4096; o->tile_out = 4096; break;
        case 8: o->block_b = 256; o->tile_in = 8192; break;
        case 9: o->log2_transform = 40; break;
        case 10: o->fd_mode = 3; break;
        case 11: o->seg_cap_gib = 1; o->fd_mode = 2; break;
        case 12: o->max_slots = 4; o->ntt_prime = 29; break;
        default: break;
    }
    return v;
}

static int query(uint64_t n, uint64_t m, int path, int v, long *ok, long *refused) {
    pa_opts o;
    memset(&o, 0, sizeof(o));
    o.device = -1;
    o.path = path;
    variant(&o, v);
    pa_plan_desc *d = (pa_plan_desc *)malloc(sizeof(pa_plan_desc));
    const int rc = pa_plan_query(n, m, &o, d);
    if (rc == PA_OK) {
        ++*ok;
        if (d->n != n || d->m != m || d->kernels_per_call == 0) {
            printf("FAIL n=%llu m=%llu path=%d v=%d\n", (unsigned long long)n,
                   (unsigned long long)m, path, v);
            free(d);
            return 1;
        }
    } else {
        ++*refused;
    }
    free(d);
    return 0;
}

int main(void) {
    static const uint64_t shapes[][2] = {
        {1, 1}, {1, 1000}, {1000, 1}, {64, 64}, {4097, 4095}, {100003, 25000},
        {1000000, 10000}, {1000000, 500000}, {2000007, 600003}, {100000007, 10000000},
        {167772160, 16000000}, {1000000007, 100000000}};
    long ok = 0, refused = 0;
    for (unsigned s = 0; s < sizeof(shapes) / sizeof(shapes[0]); ++s)
        for (int path = PA_PATH_AUTO; path <= PA_PATH_BLOCK_FP8 + 1; ++path)
            for (int v = 0; v <= 12; ++v)
                if (query(shapes[s][0], shapes[s][1], path, v, &ok, &refused)) return 1;
    /* paper-scale keys: the default plans, and the two forced plans that are refused
       before any work list is built */
    const uint64_t n = 10000000019ull, m = 1000000000ull;
    const int big[][2] = {{PA_PATH_AUTO, 0}, {PA_PATH_NTT31, 3}, {PA_PATH_NTT31, 6},
                          {PA_PATH_NTT64, 3}, {PA_PATH_NTT64, 6}};
    for (unsigned i = 0; i < sizeof(big) / sizeof(big[0]); ++i)
        if (query(n, m, big[i][0], big[i][1], &ok, &refused)) return 1;
    /* the largest sizes the interface accepts (2^40 bits): every path and option family
       plans or refuses at once, with no overflow in the geometry arithmetic */
    const uint64_t T = (uint64_t)1 << 40;
    const uint64_t edge[][2] = {{T, 1}, {1, T}, {T, T}, {T, T / 10}, {T - 1, 64}, {64, T - 1},
                                {T / 2, T / 2}, {(uint64_t)1 << 36, (uint64_t)1 << 33}};
    for (unsigned s = 0; s < sizeof(edge) / sizeof(edge[0]); ++s)
        for (int path = PA_PATH_AUTO; path <= PA_PATH_BLOCK_FP8; ++path)
            for (int v = 0; v <= 12; ++v)
                if (query(edge[s][0], edge[s][1], path, v, &ok, &refused)) return 1;
    /* invalid sizes */
    pa_plan_desc d;
    if (pa_plan_query(0, 5, NULL, &d) == PA_OK || pa_plan_query(5, 0, NULL, &d) == PA_OK ||
        pa_plan_query(5, 5, NULL, NULL) == PA_OK ||
        pa_plan_query((uint64_t)1 << 41, 5, NULL, &d) == PA_OK) {
        printf("FAIL invalid sizes accepted\n");
        return 1;
    }
    /* Eq. 1's matrix bits to the seed string, on buffers of exactly the stated sizes */
    static const uint64_t lens[] = {1, 2, 31, 32, 33, 64, 65, 1000, 4097};
    for (unsigned i = 0; i < sizeof(lens) / sizeof(lens[0]); ++i) {
        const uint64_t nn = lens[i], w = (2 * nn - 1 + 63) / 64;
        uint64_t *t = (uint64_t *)malloc(w * 8), *sd = (uint64_t *)malloc(w * 8);
        for (uint64_t k = 0; k < w; ++k) t[k] = 0x9E3779B97F4A7C15ull * (k + 1);
        if (pa_seed_from_eq1(nn, t, sd) != PA_OK) { printf("FAIL eq1 %llu\n", (unsigned long long)nn); return 1; }
        free(t);
        free(sd);
    }
    double bound = 0;
    for (uint32_t k = 5; k <= 24; ++k)
        for (int fp64 = 0; fp64 < 2; ++fp64)
            pa_fft_rounding_bound(k, (uint64_t)1 << (k - 1), (uint64_t)1 << (k - 2), fp64, &bound);
    printf("ok %ld plans, %ld refused, version %d\n", ok, refused, pa_version());
    return 0;
}
'''


def _run(cmd, **kw):
    return subprocess.run(cmd, capture_output=True, text=True, **kw)


def _gcc_can(flags, tmp):
    src = tmp / "probe.c"
    src.write_text("int main(void) { return 0; }\n")
    r = _run(["gcc"] + flags + [str(src), "-o", str(tmp / "probe")])
    return r.returncode == 0


def _build_oracle(tmp, src_text, flags, name):
    d = tmp / name
    d.mkdir()
    (d / "pa_oracle.c").write_text(src_text)
    (d / "driver.c").write_text(ORACLE_DRIVER)
    exe = d / "driver"
    r = _run(["gcc", "-std=c11", "-g", "-O1", "-pthread", "-fno-omit-frame-pointer"] + flags +
             [str(d / "pa_oracle.c"), str(d / "driver.c"), "-o", str(exe)])
    assert r.returncode == 0, r.stderr
    return exe


ASAN = ["-fsanitize=address", "-fsanitize=undefined", "-fno-sanitize-recover=all"]


@pytest.fixture(scope="module")
def oracle_text():
    with open(ORACLE_SRC) as f:
        return f.read()


def test_oracle_under_asan_ubsan(tmp_path, oracle_text):
    if not shutil.which("gcc") or not _gcc_can(ASAN, tmp_path):
        pytest.skip("gcc with AddressSanitizer is not available")
    exe = _build_oracle(tmp_path, oracle_text, ASAN, "asan")
    r = _run([str(exe)], env=SAN_ENV, timeout=600)
    assert r.returncode == 0 and "ok 13 shapes" in r.stdout, r.stdout + r.stderr[-4000:]


def test_oracle_threads_under_tsan(tmp_path, oracle_text):
    flags = ["-fsanitize=thread"]
    if not shutil.which("gcc") or not _gcc_can(flags, tmp_path):
        pytest.skip("gcc with ThreadSanitizer is not available")
    exe = _build_oracle(tmp_path, oracle_text, flags, "tsan")
    r = _run([str(exe)], env=SAN_ENV, timeout=600)
    if "unexpected memory mapping" in r.stderr or "FATAL: ThreadSanitizer" in r.stderr:
        pytest.skip("ThreadSanitizer cannot map its shadow memory on this kernel")
    assert r.returncode == 0 and "ok 13 shapes" in r.stdout, r.stdout + r.stderr[-4000:]


def test_planted_overread_is_reported(tmp_path, oracle_text):
    # the key copy reads one word past the key buffer: the instrumented oracle must report it
    if not shutil.which("gcc") or not _gcc_can(ASAN, tmp_path):
        pytest.skip("gcc with AddressSanitizer is not available")
    right = "memcpy(k, key, w * sizeof(uint64_t));"
    assert oracle_text.count(right) == 1
    planted = oracle_text.replace(right, "memcpy(k, key, (w + 1) * sizeof(uint64_t));")
    planted = planted.replace("uint64_t *k = (uint64_t *)malloc(w * sizeof(uint64_t));",
                              "uint64_t *k = (uint64_t *)malloc((w + 1) * sizeof(uint64_t));")
    exe = _build_oracle(tmp_path, planted, ASAN, "planted")
    r = _run([str(exe)], env=SAN_ENV, timeout=600)
    assert r.returncode != 0 and "heap-buffer-overflow" in r.stderr, r.stdout + r.stderr[-2000:]


@pytest.fixture(scope="module")
def san_lib(tmp_path_factory):
    """Every csrc/*.cu with host-side ASan + UBSan (device code as PTX only), as one library."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = tmp_path_factory.mktemp("plansan")
    if not os.path.exists(nvcc) or not shutil.which("gcc") or not _gcc_can(ASAN, tmp):
        pytest.skip("nvcc or gcc with AddressSanitizer is not available")
    host = "-fPIC,-fsanitize=address,-fsanitize=undefined,-fno-sanitize-recover=all," \
           "-fno-omit-frame-pointer,-g,-O1"

    def compile_one(src):
        obj = tmp / (os.path.basename(src) + ".o")
        r = _run([nvcc, "-gencode", "arch=compute_103a,code=compute_103a", "-std=c++17",
                  "--expt-relaxed-constexpr", "-Xcicc", "-O1", "-I", INCLUDE, "-Xcompiler", host,
                  "-c", src, "-o", str(obj)])
        assert r.returncode == 0, r.stderr[-3000:]
        return str(obj)

    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    lib = tmp / "libpa_san.so"
    r = _run([nvcc, "-gencode", "arch=compute_103a,code=compute_103a", "-shared",
              "-Xcompiler", "-fsanitize=address,-fsanitize=undefined", "-o", str(lib)] + objs)
    assert r.returncode == 0, r.stderr[-3000:]
    return lib


@pytest.fixture(scope="module")
def planner_exe(san_lib):
    tmp = san_lib.parent
    (tmp / "driver.c").write_text(PLANNER_DRIVER)
    exe = tmp / "driver"
    r = _run(["gcc", "-g", "-O1"] + ASAN + ["-I", INCLUDE, str(tmp / "driver.c"), str(san_lib),
              "-Wl,-rpath," + str(tmp), "-o", str(exe)])
    assert r.returncode == 0, r.stderr
    return exe


def test_planner_under_asan_ubsan(planner_exe):
    r = _run([str(planner_exe)], env=SAN_ENV, timeout=900)
    assert r.returncode == 0 and r.stdout.startswith("ok "), r.stdout[-2000:] + r.stderr[-6000:]
    ok, refused = int(r.stdout.split()[1]), int(r.stdout.split()[3])
    assert ok > 300 and refused > 100


def test_work_list_builder_under_asan_ubsan(san_lib):
    # The persistent kernel's work-list builder for batches of many blocks and small slot
    # counts (reached by no single-block query): the replay program of
    # test_work_lists.py, linked against the instrumented library, over its fixed cases
    # and a shorter random sweep.
    import test_work_lists as wl
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    tmp = san_lib.parent
    src, exe = tmp / "check.cu", tmp / "check"
    src.write_text(wl.CHECKER)
    r = _run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1",
              "-gencode", "arch=compute_103a,code=compute_103a", "-I", INCLUDE, "-I", CSRC,
              "-Xcompiler", "-fsanitize=address,-fsanitize=undefined,-fno-sanitize-recover=all,-g",
              "-Xlinker", "-rpath=" + str(tmp), str(src), str(san_lib), "-o", str(exe)])
    assert r.returncode == 0, r.stderr[-3000:]
    cases = wl._cases() + wl._random_cases(40, 77)
    run = _run([str(exe)], input=cases, env=SAN_ENV, timeout=1200)
    tail = run.stdout.splitlines()[-1] if run.stdout else ""
    assert run.returncode == 0 and tail.endswith("fails 0"), run.stdout[-2000:] + run.stderr[-6000:]
