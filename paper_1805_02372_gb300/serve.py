"""Serving driver: replays a Poisson stream of PA requests against the native server.

Requests arrive "from reconciliation by device memory": every request's key and seed are
resident on the GPU before the replay starts (Sec. 3: the corrected keys stay on the
GPU). The replay submits each request at its arrival time and polls the server, which
admits waiting requests into waves as stream slots and memory free up (continuous
batching, implemented in ``csrc/serve.cu``). Latency = completion seen by the poll -
arrival time. Only timing and bookkeeping live here; hashing is the library's.
"""
from __future__ import annotations

import time

import numpy as np

from . import binding, inputs


class Request:
    __slots__ = ("arrival", "block", "key", "seed", "out", "done", "status")

    def __init__(self, arrival, block, key, seed, out):
        self.arrival, self.block, self.key, self.seed, self.out = arrival, block, key, seed, out
        self.done = None
        self.status = None


def make_requests(count: int, rate_hz: float, device="cuda", master: int = inputs.SERVE_MASTER,
                  n_hi: float = 1e8):
    """Device-resident requests of the serving workload (Poisson arrivals)."""
    import torch
    reqs = []
    for t, b in inputs.serving_requests(count, rate_hz, master=master, n_hi=n_hi):
        k = torch.from_numpy(b.key().view(np.int64)).to(device)
        s = torch.from_numpy(b.seed().view(np.int64)).to(device)
        o = torch.zeros((b.m + 63) // 64, dtype=torch.int64, device=device)
        reqs.append(Request(t, b, k, s, o))
    torch.cuda.synchronize()
    return reqs


def at_rate(reqs, rate_hz: float, made_at_hz: float):
    """The same requests (same buffers and shapes) with their Poisson arrival times
    rescaled from the rate they were drawn at to ``rate_hz``."""
    k = made_at_hz / rate_hz
    return [Request(r.arrival * k, r.block, r.key, r.seed, r.out) for r in reqs]


def replay(reqs, slots: int = 2, max_blocks_per_wave: int = 64, memory_budget_bytes: int = 0,
           timeout_s: float = 120.0) -> dict:
    """Submit each request at its arrival time; poll until all complete."""
    srv = binding.pa_server_create(slots, max_blocks_per_wave, memory_budget_bytes)
    stats = None
    try:
        t0 = time.perf_counter()
        nxt = 0
        left = len(reqs)
        while left:
            now = time.perf_counter() - t0
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                r = reqs[nxt]
                binding.pa_server_submit(srv, r.block.n, r.block.m, r.seed, r.key, r.out, nxt)
                nxt += 1
            for tag, st in binding.pa_server_poll(srv):
                reqs[tag].done = time.perf_counter() - t0
                reqs[tag].status = st
                left -= 1
            if now > timeout_s:
                raise TimeoutError(f"{left} requests unfinished after {timeout_s} s")
        stats = binding.pa_server_get_stats(srv)
    finally:
        binding.pa_server_destroy(srv)
    lat = np.array([(r.done - r.arrival) * 1e3 for r in reqs])
    span = max(r.done for r in reqs) - reqs[0].arrival
    bits = sum(r.block.n for r in reqs)
    offered = bits / max(reqs[-1].arrival - reqs[0].arrival, 1e-9)
    q = max(1, len(reqs) // 4)
    waves = max(1, stats["waves"])
    return {"requests": len(reqs), "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "max_ms": float(lat.max()),
            "sustained_gbps": bits / span / 1e9, "offered_gbps": offered / 1e9,
            "errors": sum(1 for r in reqs if r.status != 0),
            # latency drift: median of the last quarter of arrivals over the first quarter's
            # (well above 1 when the queue grows, i.e. past saturation)
            "latency_drift": float(np.median(lat[-q:]) / max(np.median(lat[:q]), 1e-9)),
            "waves": stats["waves"], "waves_held_back": stats["waves_held_back"],
            "host_plan_ms_per_wave": stats["plan_s_total"] / waves * 1e3,
            "host_plan_ms_max": stats["plan_s_max"] * 1e3}
