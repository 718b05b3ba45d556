"""Multi-rank host logic on CPU (gloo, world size 2): reductions and failure detection."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, scenario, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    from paper_1805_02372_gb300.dist import Group, RankFailure
    g = Group("gloo", rank, world, timeout_s=20)
    try:
        if scenario == "reduce":
            q.put((rank, g.max((rank + 1) * 1.5), g.sum((rank + 1) * 1.5)))
            g.checked_barrier("done", 10)
        elif scenario == "fail":
            if rank == 1:
                g.report_failure("step", "RuntimeError: injected on the host")
                q.put((rank, "reported"))
                return
            try:
                g.checked_barrier("step", 10)
                q.put((rank, "no error"))
            except RankFailure as e:
                q.put((rank, f"RankFailure: {e}"))
        elif scenario == "vanish":
            if rank == 1:
                q.put((rank, "exited"))
                return
            try:
                g.checked_barrier("step", 2)
                q.put((rank, "no error"))
            except RankFailure as e:
                q.put((rank, f"RankFailure: {e}"))
    finally:
        if scenario == "reduce":
            g.close()


def _run(scenario):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, scenario, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = dict()
    for _ in range(2):
        r, *v = q.get(timeout=60)
        out[r] = v
    for p in procs:
        p.join(timeout=30)
        if p.is_alive():
            p.kill()
    return out


def test_max_and_sum_over_ranks():
    out = _run("reduce")
    assert out[0] == [3.0, 4.5] and out[1] == [3.0, 4.5]


def test_rank_failure_reported_on_host():
    out = _run("fail")
    assert out[1] == ["reported"]
    assert out[0][0].startswith("RankFailure") and "injected" in out[0][0]


def test_missing_rank_times_out():
    out = _run("vanish")
    assert out[0][0].startswith("RankFailure") and "did not reach" in out[0][0]
