"""FFT path: bit-exact output and a measured worst residual below the proven bound."""
import numpy as np
import pytest

import oracle
import paper_1805_02372_gb300 as pkg
from paper_1805_02372_gb300 import inputs
from gpu_util import dev, host

pytestmark = pytest.mark.gpu


def _run(n, m, key, seed, **opts):
    import torch
    plan = pkg.Plan(n, m, path="fft", **opts)
    out = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
    plan.hash(dev(seed), dev(key), out)
    torch.cuda.synchronize()
    res, bound = plan.residual()
    desc = plan.desc
    plan.close()
    return host(out), res, bound, desc


@pytest.mark.parametrize("kind", ["random", "ones"])
@pytest.mark.parametrize("n,m", [(100_003, 25_000), (20_000, 7_777)])
def test_residual_below_bound(kind, n, m):
    if kind == "ones":
        key = np.full((n + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
        seed = np.full((n + m - 1 + 63) // 64, np.uint64(0xFFFFFFFFFFFFFFFF))
    else:
        b = inputs.single_block(n, m, 31, 32)
        key, seed = b.key(), b.seed()
    got, res, bound, desc = _run(n, m, key, seed)
    assert np.array_equal(got, oracle.hash_full(n, m, seed, key))
    assert desc["fp64"] == 0 and bound == desc["rounding_bound"] < 0.5
    assert 0.0 <= res <= bound, (res, bound)


def test_fp64_on_lengths_where_fp32_fails():
    n, m = 50_000, 9_000
    b = inputs.single_block(n, m, 41, 42)
    key, seed = b.key(), b.seed()
    got, res, bound, desc = _run(n, m, key, seed, log2_transform=12, tile_in=2048,
                                 tile_out=2048)
    assert desc["fp64"] == 1
    assert np.array_equal(got, oracle.hash_full(n, m, seed, key))
    assert res <= bound < 1e-8
