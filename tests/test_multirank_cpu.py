"""The N > 1 host path of bench.py on CPU: two gloo ranks (one process each,
rendezvous on 127.0.0.1), as torchrun would start them on two GPUs.

Checks the parts that need no GPU: every rank agrees on the slowest rank's
time, the whole-job throughput counts all ranks' pixels over that time, each
rank filters its own seeded image (replicas are independent), and the
reference arm prints from rank 0 only.
"""
import io
import json
import os
import socket
import contextlib

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 10.0 + 5.0 * rank          # rank 1 is the slow one
        slowest = bench.max_over_ranks(local_ms, world, "cpu")
        value = bench.replica_throughput(4.0e6, 3, world, slowest)
        w = bench._workload("c1", rank)
        digest = float(np.asarray(w["image"], dtype=np.float64).sum())
        out = io.StringIO()
        args = type("A", (), dict(workload="c1", steps=1, warmup=0))()
        if rank != 0:
            with contextlib.redirect_stdout(out):
                bench.run_reference(args)
        dist.barrier()
        q.put((rank, slowest, value, digest, out.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_replicas():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    assert [r[1] for r in res] == [15.0, 15.0]            # max over ranks, on every rank
    assert res[0][2] == pytest.approx(4.0e6 * 3 * 2 / 15e-3 / 1e6)
    assert res[0][3] != res[1][3]                          # each replica its own image
    assert res[1][4] == ""                                 # reference arm: rank 1 prints nothing


def test_single_rank_helpers_are_identity():
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.replica_throughput(1e6, 10, 1, 1000.0) == pytest.approx(10.0)
