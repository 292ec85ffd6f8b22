"""Host side of the multi-GPU benchmark: the method's independent instances run as
replicas, one per rank (no exchange on the data path).  The only collectives are a
barrier around the timed region and a max over ranks of the elapsed time; the job's
throughput is every rank's solves divided by the slowest rank's time ("weak" scaling).
Backend-agnostic, so the same code is exercised with gloo on CPU in the tests and with
NCCL on GPUs in the benchmark."""
from __future__ import annotations

import os


def env():
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier(ws: int):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, ws: int, device=None) -> float:
    if ws == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(ms_per_step_max: float, ws: int, solves_per_step: int = 1) -> float:
    """Solves per second of the whole job: all ranks' solves over the slowest rank's time."""
    return ws * solves_per_step * 1e3 / ms_per_step_max
