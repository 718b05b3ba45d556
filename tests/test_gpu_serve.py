"""Serving: continuous batching returns, for every request, the same bits as the oracle
and as the request hashed alone; latency statistics are reported."""
import numpy as np
import pytest

import oracle
import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import serve
from gpu_util import host

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("rate,slots", [(2000.0, 2), (200.0, 3)])
def test_each_result_same_alone_and_in_the_mix(rate, slots):
    import torch
    reqs = serve.make_requests(40, rate, n_hi=3e6)
    stats = serve.replay(reqs, slots=slots, max_blocks_per_wave=16)
    assert stats["errors"] == 0 and stats["p50_ms"] <= stats["p99_ms"]
    for r in reqs:
        b = r.block
        got = host(r.out)
        # alone: one plan, one call
        plan = pkg.Plan(b.n, b.m)
        o = torch.zeros_like(r.out)
        plan.hash(r.seed, r.key, o)
        torch.cuda.synchronize()
        plan.close()
        assert np.array_equal(host(o), got), (b.n, b.m)
    # and the oracle on a sample of requests
    for r in reqs[::8]:
        b = r.block
        assert np.array_equal(oracle.hash_full(b.n, b.m, b.seed(), b.key()), host(r.out))


def test_memory_budget_admission():
    reqs = serve.make_requests(12, 5000.0, n_hi=2e6, master=9)
    stats = serve.replay(reqs, slots=4, max_blocks_per_wave=4, memory_budget_bytes=64 << 20)
    assert stats["errors"] == 0
    for r in reqs[::3]:
        b = r.block
        assert np.array_equal(oracle.hash_full(b.n, b.m, b.seed(), b.key()), host(r.out))
