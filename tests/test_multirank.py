"""The N-replica path of bench.py on CPU: two gloo ranks (one process each,
127.0.0.1 rendezvous) reduce their step times to the slowest rank's and report
whole-job rates over all ranks' keys; the reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # per-rank (total, build, query) ms: rank 1 is slower at building, rank 0 at querying
        mine = [100.0 + rank, 40.0 + 5.0 * rank, 9.0 - rank]
        got = bench.reduce_max(mine, dist, "cpu")
        q.put((rank, got, bench.job_rates(got[1], got[2], 1_000_000, world)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_aggregate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, (ns, gq) in res:
        assert got == [101.0, 45.0, 9.0]  # element-wise max over ranks
        # 2 replicas x 1e6 keys in 45 ms -> 22.5 ns/key; 2 x 2e6 queries in 9 ms
        assert ns == pytest.approx(45.0e6 / 2e6) and gq == pytest.approx(4e6 / 9e-3 / 1e9)


def test_single_rank_rates_and_reference_arm_rank_gate(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    assert bench.reduce_max([1, 2.5], None, "cpu") == [1.0, 2.5]
    ns, gq = bench.job_rates(80.0, 4.0, 10**8, 1)
    assert ns == pytest.approx(0.8) and gq == pytest.approx(50.0)
    # under torchrun only rank 0 times the oracle; the others leave without work
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")

    class A:
        workload, steps, warmup = "c2", 1, 0

    assert bench.run_reference(A()) is None
