"""The no-allocation entry point (pa_hash_direct_static) against the planned one and the oracle.

Callers that cannot allocate device memory (a pipeline that reserved its memory once at
start-up, a process whose device memory belongs to another allocator) use the entry point
whose scratch is a fixed static array. Its output must equal pa_hash's on the direct path
and the CPU oracle's, bit for bit, on two calls in a row (the second smaller, so stale
scratch from the first call would show), up to the documented key-length limit n = 2^25;
free device memory must not move across a call; the status call must read PA_OK after a
normal run. This file is collected last, so a failure here stops a -x run only after every
other test ran.
"""
import numpy as np
import pytest

import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding, inputs
from gpu_util import dev, host

pytestmark = pytest.mark.gpu

STATIC_MAX_N = 1 << 25


def _static_vs_planned_vs_oracle(oracle, n, m, ks):
    import torch
    b = inputs.single_block(n, m, ks, ks + 1)
    key_h, seed_h = b.key(), b.seed()
    seed, key = dev(seed_h), dev(key_h)
    got = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
    pkg.binding.pa_hash_direct_static(n, m, seed, key, got)
    assert pkg.binding.pa_direct_static_status() == binding.PA_OK
    plan = pkg.Plan(n, m, path="direct")
    want = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
    plan.hash(seed, key, want)
    torch.cuda.synchronize()
    plan.close()
    g = host(got)
    assert np.array_equal(g, host(want)), (n, m)
    assert np.array_equal(g, oracle.hash_full(n, m, seed_h, key_h)), (n, m)


def test_static_scratch_entry_matches_planned_entry_and_oracle(oracle):
    # two calls in a row, the second smaller (stale scratch from the first would show)
    for n, m, ks in [(1_000_003, 250_001, 61), (100_003, 25_000, 63)]:
        _static_vs_planned_vs_oracle(oracle, n, m, ks)


def test_static_scratch_at_its_limit(oracle):
    # the largest key the static array holds, then a small one after it
    _static_vs_planned_vs_oracle(oracle, STATIC_MAX_N, 1_000, 65)
    _static_vs_planned_vs_oracle(oracle, 4_097, 77, 67)


def test_static_scratch_allocates_nothing():
    import torch
    n, m = 2_000_003, 100_000
    b = inputs.single_block(n, m, 69, 70)
    seed, key = dev(b.seed()), dev(b.key())
    out = torch.zeros(((m + 63) // 64,), dtype=torch.int64, device="cuda")
    pkg.binding.pa_hash_direct_static(n, m, seed, key, out)  # first call on the device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pkg.binding.pa_hash_direct_static(n, m, seed, key, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert pkg.binding.pa_direct_static_status() == binding.PA_OK


def test_static_scratch_rejects_oversize():
    import torch
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(pkg.PAError) as e:
        pkg.binding.pa_hash_direct_static(STATIC_MAX_N + 1, 10, buf, buf, buf)
    assert e.value.status == binding.PA_ERR_TOO_LARGE
