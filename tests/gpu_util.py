"""Helpers for the GPU tests: device buffers and one call through the C ABI."""
import numpy as np

import paper_1805_02372_gb300 as pkg


def dev(words: np.ndarray):
    import torch
    return torch.from_numpy(np.ascontiguousarray(words, dtype=np.uint64).view(np.int64)).cuda()


def host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def run_path(n, m, key, seed, path="auto", **opts):
    """Hash on the GPU through pa_plan_ex + pa_hash; output buffer prefilled with ones."""
    import torch
    plan = pkg.Plan(n, m, path=path, **opts)
    try:
        out = torch.full(((m + 63) // 64,), -1, dtype=torch.int64, device="cuda")
        plan.hash(dev(seed), dev(key), out)
        torch.cuda.synchronize()
        st = plan.status()
        assert st == 0, f"device status {st}"
        return host(out), plan.desc
    finally:
        plan.close()
