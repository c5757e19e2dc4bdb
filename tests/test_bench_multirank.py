"""The N > 1 host logic of bench.py on CPU: two gloo ranks (one process per
rank, as torchrun starts them).  Each rank decodes its own frame, so the
job's value is the sum of the ranks' clusters over the slowest rank's time;
ranks get different input seeds; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r decodes 1000 (r + 1) clusters in 0.5 (r + 1) s
        rate = bench.whole_job_rate(1000.0 * (rank + 1), 0.5 * (rank + 1))
        slowest = bench._reduce(0.5 * (rank + 1), "max")
        total = bench._reduce(1000.0 * (rank + 1), "sum")
        q.put((rank, rate, slowest, total, bench._dist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_job():
    pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, rate, slowest, total, dist in res:
        assert slowest == 1.0 and total == 3000.0
        assert rate == pytest.approx(3000.0)           # (1000 + 2000) / max(0.5, 1.0)
        assert dist == (2, rank, rank)


def test_single_process_reduces_to_itself():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(123.0, 2.0) == pytest.approx(61.5)


def test_ranks_decode_different_frames(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    (t0, s0), (t1, s1) = bench.make_inputs(0, scale=0.0005), bench.make_inputs(1, scale=0.0005)
    assert s1 == s0 + 1
    assert len(t0["row"]) != len(t1["row"]) or (t0["row"] != t1["row"]).any()


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        steps, warmup = 1, 0
    assert bench.run_reference(A()) == 0
