"""The multi-rank benchmark path (replicas of independent instances) on CPU: two gloo
ranks over 127.0.0.1 exercise the barrier, the max over ranks of the timed region and the
job throughput exactly as the NCCL ranks of the benchmark do."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    from paper_2406_15959_gb300 import replicas as R
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, lr = R.env()
        assert (w, r, lr) == (ws, rank, rank)
        R.barrier(w)
        ms_local = 100.0 + 50.0 * rank          # the slower rank sets the job's time
        ms = R.max_over_ranks(ms_local, w)
        out[rank] = (ms, R.job_throughput(ms, w))
        R.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1] == (150.0, 2 * 1e3 / 150.0)


def test_single_rank_needs_no_process_group():
    from paper_2406_15959_gb300 import replicas as R
    R.barrier(1)
    assert R.max_over_ranks(3.5, 1) == 3.5
    assert R.job_throughput(250.0, 1) == 4.0
