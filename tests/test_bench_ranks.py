"""Multi-process path of bench.py on CPU: two gloo ranks.  The job's time is
the slowest rank's, the job's rate counts every rank's work, and the
reference arm runs on rank 0 only (replicas only: no data-path collective)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}")
    try:
        slowest = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu")
        rate = bench.job_rate(4, world, slowest)
        ref = bench.reference_arm(type("A", (), {"warmup": 0, "steps": 0, "workload": "L128_b6_massweep",
                                                 "oracle_iters": 0})()) if rank == 1 else None
        out.put((rank, slowest, rate, ref))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_job_rate():
    ctx = torch.multiprocessing.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, slowest, rate, ref in res:
        assert slowest == 15.0                  # the slowest rank's time, on every rank
        assert rate == pytest.approx(4 * 2 / 15.0)
        assert ref is None                      # the reference arm does no work off rank 0


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(4, 1, 2.0) == 2.0
