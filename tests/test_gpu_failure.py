"""Failure detection on the GPU without a fault: bounded waits that can never be satisfied
return PA_ERR_TIMEOUT through the status word, and the context keeps working."""
import numpy as np
import pytest

import oracle
import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import binding, inputs
from gpu_util import run_path

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [1, 2])
def test_bounded_wait_reports_timeout(which):
    import time
    t0 = time.perf_counter()
    assert pkg.binding.pa_selftest(which) == binding.PA_ERR_TIMEOUT
    # the wait is bounded in time (4 s, plus at most 0.5 s of draining), not in polls
    assert 3.5 < time.perf_counter() - t0 < 15.0
    # the context is still usable: a hash right after is bit-exact
    b = inputs.single_block(50_001, 7_777, 91, 92)
    got, _ = run_path(b.n, b.m, b.key(), b.seed(), path="auto")
    assert np.array_equal(got, oracle.hash_full(b.n, b.m, b.seed(), b.key()))


def test_status_clean_after_normal_runs():
    import torch
    b = inputs.single_block(200_003, 60_001, 93, 94)
    plan = pkg.Plan(b.n, b.m, path="ntt31")
    from gpu_util import dev
    out = torch.zeros((b.m + 63) // 64, dtype=torch.int64, device="cuda")
    plan.hash(dev(b.seed()), dev(b.key()), out)
    assert plan.status() == 0
    plan.close()
