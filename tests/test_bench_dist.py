"""The multi-rank aggregation of bench.py on CPU ranks (gloo, world size 2).

Each rank times its own replica; the bench reports every rank's bytes over
the slowest rank's time.  Two processes with different local times check the
max-over-ranks and the whole-job rate the GPU bench uses (there on NCCL)."""

import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        local_ms = 10.0 + 5.0 * rank            # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, "cpu")
        rate = bench.whole_job_rate(w, 1e9, ms)
        out.put((r, w, local, ms, rate))
    finally:
        dist.destroy_process_group()


def test_bench_aggregates_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, (r, w, local, ms, rate) in enumerate(res):
        assert (r, w, local) == (rank, 2, rank)
        assert ms == 15.0                          # the slower rank's time on both
        assert rate == pytest.approx(2 * 1e9 / 15e-3 / 1e9)


def test_single_process_keeps_its_own_time():
    import bench
    assert bench.max_over_ranks(3.5, "cpu") == 3.5
    assert bench.whole_job_rate(1, 2e9, 1000.0) == pytest.approx(2.0)
