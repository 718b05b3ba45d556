"""The no-allocation entry point (pa_hash_direct_static) against the planned one.

Callers that cannot allocate device memory (a pipeline that reserved its memory once at
start-up, a process whose device memory belongs to another allocator) use the entry point
whose scratch is a fixed static array. Its output must equal pa_hash's on the direct path,
bit for bit, on two calls in a row (the second smaller, so stale scratch from the first
call would show).
"""
import numpy as np
import pytest

import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding, inputs
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def test_static_scratch_entry_matches_planned_entry():
    import torch
    for n, m, ks in [(1_000_003, 250_001, 61), (100_003, 25_000, 63)]:
        b = inputs.single_block(n, m, ks, ks + 1)
        seed, key = dev(b.seed()), dev(b.key())
        got = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
        pkg.binding.pa_hash_direct_static(n, m, seed, key, got)
        plan = pkg.Plan(n, m, path="direct")
        want = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
        plan.hash(seed, key, want)
        torch.cuda.synchronize()
        plan.close()
        assert np.array_equal(host(got), host(want)), (n, m)


def test_static_scratch_rejects_oversize():
    import torch
    buf = torch.zeros(16, dtype=torch.int64, device="cuda")
    with pytest.raises(pkg.PAError) as e:
        pkg.binding.pa_hash_direct_static((1 << 25) + 1, 10, buf, buf, buf)
    assert e.value.status == binding.PA_ERR_TOO_LARGE
