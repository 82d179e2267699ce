"""The N > 1 path of the benchmark is replicas only (each rank steps its own
lattice, no data exchange): its host logic -- the slowest rank's time as the
job's time, and the whole-job rate over all ranks' site updates -- runs here on
two gloo ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench

        ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
        job_ms = bench.max_over_ranks(ms, "cpu")
        q.put((rank, job_ms, bench.whole_job_mlups(1000, 10, world, job_ms)))
    finally:
        dist.destroy_process_group()


def test_two_rank_replica_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 2000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[1] for g in got] == [150.0, 150.0]
    # 2 replicas x 1000 sites x 10 steps in 150 ms
    assert got[0][2] == pytest.approx(2 * 1000 * 10 / 0.150 / 1e6)
    assert got[0][2] == got[1][2]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    called = []
    monkeypatch.setattr(bench, "fields", lambda: called.append(1))
    bench.run_reference(type("A", (), {"warmup": 0, "steps": 1})(), rank=1, world=2)
    assert called == []
