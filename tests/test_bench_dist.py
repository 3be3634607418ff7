"""The bench's multi-process path on the host: N independent replicas (the probe path shards by
volume with no exchange), a barrier, the max of the ranks' times, the whole-job value, and the
reference arm running on rank 0 only. world_size 2 over gloo, as the GPU runs use NCCL."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import argparse

    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (ws, rank) and dist.get_backend() == "gloo"
    bench.barrier(w)
    t_max = bench.max_over_ranks(10.0 + rank, w)               # the slowest rank decides
    value = bench.job_value(4096, 60, w, t_max)
    # the reference arm: ranks other than 0 leave without work
    args = argparse.Namespace(steps=1, warmup=0, gpus=w)
    if rank != 0:
        bench.run_reference(args, w, rank)
    bench.barrier(w)
    out.put((rank, t_max, value))
    dist.destroy_process_group()


def test_two_replicas_take_the_max_and_count_every_rank():
    ws = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(out.get(timeout=5) for _ in range(ws))
    for rank, t_max, value in got:
        assert t_max == 10.0 + (ws - 1)
        assert value == pytest.approx(4096 * 60 * ws / ((10.0 + ws - 1) / 1e3))
