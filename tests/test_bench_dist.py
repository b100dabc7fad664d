"""The multi-process path of bench.py on the CPU: two gloo ranks (the GPU runs
are replicas, one field per rank, with no data-path collective; only the
timing takes the maximum over ranks)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    try:
        import bench
        dist.init_process_group("gloo", rank=rank, world_size=world)
        try:
            w, r, _ = bench.dist_setup()
            slowest = bench.max_over_ranks(100.0 + 10.0 * r, w, torch.device("cpu"))
            value = bench.job_throughput(1000, w, slowest)
            # each rank integrates its own field (seed + rank): replicas, weak scaling
            T, p, Y, cls = bench.states.bimodal_states(bench.NSP, bench.NRX, 64, bench.SEED + r)
            q.put((r, w, slowest, value, float(T.sum())))
        finally:
            dist.destroy_process_group()
    except Exception as e:      # report instead of leaving the parent waiting
        q.put((rank, "error", repr(e), None, None))


@pytest.mark.timeout(300)
def test_two_gloo_ranks_take_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = sorted((q.get(timeout=240) for _ in range(world)), key=lambda o: o[0])
    assert all(o[1] != "error" for o in out), out
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    assert [o[0] for o in out] == [0, 1] and all(o[1] == 2 for o in out)
    assert all(o[2] == 110.0 for o in out)                     # max over ranks, seen by every rank
    assert all(o[3] == pytest.approx(2 * 1000 / 0.110) for o in out)
    assert out[0][4] != out[1][4]                              # different fields per rank


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(42.0, 1) == 42.0
    assert bench.job_throughput(262144, 1, 1000.0) == pytest.approx(262144.0)
