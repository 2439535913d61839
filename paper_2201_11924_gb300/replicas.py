"""Independent replicas across GPUs (one process per GPU, launched by torchrun).

The depth stage has no exchange step: stereo pairs (and serving requests) are
independent, so N GPUs run N replicas, each on its own pairs (weak scaling),
and the only cross-rank operations are the timing barrier and the maximum of
the ranks' elapsed times.  NCCL carries them between GPUs; gloo carries the
same calls between CPU processes, which is how the multi-rank host logic is
tested without several GPUs.
"""
from __future__ import annotations

import os
from dataclasses import dataclass


@dataclass
class Replicas:
    world: int
    rank: int
    local: int
    backend: str | None = None   # None: single process, no process group

    @property
    def distributed(self) -> bool:
        return self.backend is not None

    def barrier(self):
        if self.distributed:
            import torch.distributed as dist
            dist.barrier()

    def max_over_ranks(self, value: float, device=None) -> float:
        """The maximum of `value` over all ranks (the job's elapsed time is
        the slowest rank's)."""
        if not self.distributed:
            return float(value)
        import torch
        import torch.distributed as dist
        dev = device if (device is not None and self.backend == "nccl") else "cpu"
        t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.distributed:
            import torch.distributed as dist
            dist.destroy_process_group()


# Seconds a collective (the barrier, the maximum) waits for the other ranks
# before it fails: a rank that died or never joins ends the others' wait with
# an error instead of the process group's default half hour.
DEFAULT_TIMEOUT_S = 300.0


def from_env(backend: str | None = None, timeout_s: float | None = None) -> Replicas:
    """Reads WORLD_SIZE / RANK / LOCAL_RANK (torchrun's variables) and, for
    more than one rank, joins the process group: NCCL when CUDA is available,
    gloo otherwise (or the given backend).  timeout_s (default: the
    SIMSENSE_COLLECTIVE_TIMEOUT_S variable, else DEFAULT_TIMEOUT_S) bounds
    every collective's wait for the other ranks."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world <= 1:
        return Replicas(1, 0, 0, None)
    import datetime

    import torch
    import torch.distributed as dist
    if backend is None:
        backend = "nccl" if torch.cuda.is_available() else "gloo"
    if backend == "nccl":
        torch.cuda.set_device(local)
    if timeout_s is None:
        timeout_s = float(os.environ.get("SIMSENSE_COLLECTIVE_TIMEOUT_S", DEFAULT_TIMEOUT_S))
    dist.init_process_group(backend, timeout=datetime.timedelta(seconds=timeout_s))
    return Replicas(world, rank, local, backend)


def shard(n_units: int, rank: int, world: int) -> list[int]:
    """Units (pairs, cameras) a rank owns: every world-th unit from rank on,
    so each rank gets n_units // world or one more and no unit is shared."""
    return list(range(rank, n_units, world))
