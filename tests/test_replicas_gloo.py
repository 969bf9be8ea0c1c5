"""Multi-process replica bookkeeping of bench.py on CPU (gloo, world size 2):
each rank draws its own seeded instances, the replica results combine as
sum of work over max of time, and only rank 0 reports.  The data path has no
collective, so nothing else needs more than one process."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    w, r, _ = bench.dist_setup(backend="gloo")
    insts, _desc = bench.make_workload("vortex2d", r)
    checksum = float(np.sum(insts[0].u0))
    bench.barrier(w)
    total = bench.reduce_over_ranks(10.0 * (r + 1), w, "sum")
    slowest = bench.reduce_over_ranks(1.0 + r, w, "max")
    import torch
    sums = [torch.zeros(1, dtype=torch.float64) for _ in range(w)]
    dist.all_gather(sums, torch.tensor([checksum], dtype=torch.float64))
    out.put((r, w, total, slowest, [float(x) for x in sums]))
    dist.destroy_process_group()


def test_two_gloo_ranks_replica_bookkeeping():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, total, slowest, sums in res:
        assert w == 2
        assert total == 30.0 and slowest == 2.0          # sum of work, max of time
        assert sums[0] != sums[1]                        # each rank has its own seeded instances


def test_reference_arm_rank_nonzero_is_silent(capsys):
    """Under torchrun only rank 0 runs and prints the reference line."""
    sys.path.insert(0, ROOT)
    import bench
    old = os.environ.get("RANK")
    os.environ["RANK"] = "1"
    try:
        class A:
            workload, steps, warmup, gpus = "burgers1d", 1, 0, 2
        bench.run_reference(A)
    finally:
        if old is None:
            del os.environ["RANK"]
        else:
            os.environ["RANK"] = old
    assert capsys.readouterr().out == ""
