"""Multi-rank coordination for replicas: one process per GPU, each hashing its own blocks.

Independent PA blocks shard across GPUs with no data-path exchange (weak scaling); the
only cross-rank traffic is timing (max over ranks), unit totals (sum) and liveness. A
rank that fails writes its error to the shared store, and every other rank learns of it
at its next checked barrier, within a timeout, instead of blocking in a collective.
"""
from __future__ import annotations

import datetime
import os
import time


class RankFailure(RuntimeError):
    pass


def env():
    """(rank, world_size, local_rank) from the launcher's environment (1 rank if unset)."""
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class Group:
    """A process group plus its TCP store (rank 0 hosts it)."""

    def __init__(self, backend: str, rank: int, world: int, timeout_s: float = 60.0,
                 device=None):
        import torch.distributed as dist
        from torch.distributed import distributed_c10d as c10d
        self.dist, self.rank, self.world, self.device = dist, rank, world, device
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        td = datetime.timedelta(seconds=timeout_s)
        kw = {"device_id": device} if (backend == "nccl" and device is not None) else {}
        # env:// works both under torchrun (its agent hosts the store) and plain env vars
        dist.init_process_group(backend, init_method="env://", rank=rank, world_size=world,
                                timeout=td, **kw)
        self.store = c10d._get_default_store()

    def _tensor(self, x):
        import torch
        return torch.tensor([float(x)], dtype=torch.float64,
                            device=self.device if self.device is not None else "cpu")

    def max(self, x: float) -> float:
        t = self._tensor(x)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        t = self._tensor(x)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        return float(t.item())

    def report_failure(self, tag: str, message: str) -> None:
        self.store.set(f"fail/{tag}/{self.rank}", message[:500])

    def checked_barrier(self, tag: str, timeout_s: float = 30.0) -> None:
        """Barrier through the store: raises RankFailure naming the ranks that reported a
        failure or did not arrive within timeout_s (never blocks longer)."""
        self.store.set(f"arrive/{tag}/{self.rank}", "1")
        deadline = time.monotonic() + timeout_s
        while True:
            failed, missing = [], []
            for r in range(self.world):
                if self.store.check([f"fail/{tag}/{r}"]):
                    failed.append((r, self.store.get(f"fail/{tag}/{r}").decode()))
                elif not self.store.check([f"arrive/{tag}/{r}"]):
                    missing.append(r)
            if failed:
                raise RankFailure(f"ranks failed at {tag}: {failed}")
            if not missing:
                return
            if time.monotonic() > deadline:
                raise RankFailure(f"ranks {missing} did not reach {tag} within {timeout_s} s")
            time.sleep(0.01)

    def close(self):
        try:
            self.dist.destroy_process_group()
        except Exception:
            pass
