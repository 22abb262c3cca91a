"""The N-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1 run the bookkeeping that
the GPU ranks run (independent replicas with distinct seeded orbitals, the slowest rank's
time, the whole-job rate over all ranks' units), with no collective on the data path."""
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


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_local = 1.0 + 0.5 * rank                     # rank 1 is the slow one
        t = bench.max_over_ranks(t_local, torch.device("cpu"))
        rate = bench.whole_job_rate(100.0, 3, world, t)
        seeds = [bench.replica_spin_index(s, rank) for s in range(2)]
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        if rank == 0:
            out.put({"t": t, "rate": rate, "seeds": gathered})
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_gpu_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert res["t"] == 1.5                              # the slowest rank's time
    assert res["rate"] == pytest.approx(100.0 * 3 * 2 / 1.5)
    flat = [s for seeds in res["seeds"] for s in seeds]
    assert len(set(flat)) == len(flat)                 # every replica starts from its own orbitals


def test_replicas_draw_distinct_orbitals():
    sys.path.insert(0, ROOT)
    import bench
    import workloads as w
    wl = w.tiny()
    a = wl.orbitals(bench.replica_spin_index(0, 0))
    b = wl.orbitals(bench.replica_spin_index(0, 1))
    assert a.shape == b.shape and not np.allclose(a, b)


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(2.5, None) == 2.5
