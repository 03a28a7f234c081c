"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): weak
scaling with one independent tensor per rank, the slowest rank's time, the
whole-job value, and the reference arm doing no work off rank 0."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2504_04989_gb300 import workloads as wl
    t_max = bench.max_over_ranks(1.0 + rank)          # rank r "took" 1 + r seconds
    value = bench.job_value(10, world, t_max)
    X = wl.make_c1(seed=rank)                           # each rank its own tensor (seed = rank)
    digest = float(np.sum(X[0, :4, :4]))
    bench.run_reference(type("A", (), {"warmup": 0, "steps": 0, "gpus": world})(), {}, rank, world) \
        if rank != 0 else None                          # off rank 0 the reference arm returns at once
    q.put((rank, t_max, value, digest))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [2.0, 2.0]            # max over ranks, seen by every rank
    assert [o[2] for o in out] == [10.0, 10.0]          # 2 ranks x 10 steps / 2 s
    assert out[0][3] != out[1][3]                       # independent tensors per rank


def test_single_process_helpers():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(20, 1, 0.5) == 40.0
