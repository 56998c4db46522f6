"""World-size-2 checks of bench.py's multi-rank logic on CPU over gloo. The transform shards as
independent replicas: every rank runs the whole batch, with no collective on the data path. The
only exchange is the timing: the job takes as long as its slowest rank, and the whole-job rate
counts every rank's outputs. The reference arm runs on rank 0 alone; the other ranks return at once.
"""
import argparse
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        env = bench.dist_setup()
        seconds = [3.0, 5.0, 4.0, 1.0][rank]  # this rank's time for its replica
        slowest = bench.max_over_ranks(seconds, ws, "cpu")
        rate = bench.job_rate(1000, ws, slowest)
        ref = "not run"
        if rank != 0:
            ref = bench.run_reference(argparse.Namespace(steps=1, warmup=0, gpus=ws), ws, rank)
        q.put((rank, env, slowest, rate, ref))
    finally:
        dist.destroy_process_group()


def _run(ws):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return res


def test_replicas_time_is_the_slowest_rank_over_gloo():
    res = _run(2)
    assert [r[0] for r in res] == [0, 1]
    for rank, env, slowest, rate, ref in res:
        assert env == (2, rank, rank)
        assert slowest == 5.0
        assert rate == 2 * 1000 / 5.0
        assert ref == ("not run" if rank == 0 else None)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_rate(1000, 1, 2.0) == 500.0
