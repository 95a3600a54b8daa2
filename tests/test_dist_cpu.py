"""The multi-GPU path is replicas only (one independent problem per rank, no
data-path collective): what N > 1 adds is host logic — a barrier around the
timed region, the slowest rank's time, and the whole-job rate.  Checked here
with world size 2 on the gloo backend, on CPU."""

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    got_env = bench.dist_env()
    dist.barrier()
    # rank r timed (r + 1) * 100 ms for 5 steps of 8 vectors
    t_max = bench.max_over_ranks(100.0 * (rank + 1), ws, torch.device("cpu"))
    value = bench.whole_job_rate(ws, 8, 5, t_max)
    out.put((rank, got_env, t_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_world_size_2():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, env, t_max, value in res:
        assert env == (ws, rank, rank)
        assert t_max == pytest.approx(200.0)  # the slowest rank
        # 2 ranks x 8 vectors x 5 steps in 0.2 s
        assert value == pytest.approx(2 * 8 * 5 / 0.2)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.max_over_ranks(123.0, 1, None) == 123.0
    assert bench.whole_job_rate(1, 8, 5, 1000.0) == pytest.approx(40.0)
