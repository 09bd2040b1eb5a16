"""The N > 1 path of bench.py with two gloo ranks on the CPU.  The
single-instance path does not shard (replicas only), so a multi-rank run has
no data-path collective: each rank runs its own simulation, the ranks agree
on the slowest rank's time (max over ranks), the whole-job rate counts every
rank's units against that time, and only rank 0 runs and prints the
reference arm."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _Args:
    workload = "film_64x16x1"
    steps = 1
    warmup = 3


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["MM_REF_BUDGET_S"] = "0.01"
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        t = (0.25, 0.75)[rank]
        t_max = bench.max_over_ranks(t, world, "cpu")
        rate = bench.whole_job_rate(1000, world, t_max)
        dist.barrier()
        out = bench.run_reference(_Args, rank, world)
        q.put((rank, t_max, rate, out is None, None if out is None else out["impl"]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t_max, rate, _, _ in res:
        assert t_max == 0.75
        assert rate == pytest.approx(2 * 1000 / 0.75)
    # rank 0 alone runs the (oracle) reference arm; rank 1 does no work
    assert res[0][3] is False and res[0][4] == "reference"
    assert res[1][3] is True


def _shard_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1406_7635_gb300.shard import gather_instance_stats, instance_shard
        n = 11
        ids = instance_shard(n, rank, world)
        # stand-ins for the stats a rank's own batch reports for its instances
        stats = [{"accepted": 100 + i, "rejected": i % 3, "t": 1e-10 + i * 1e-15, "status": -4 if i == 7 else 0}
                 for i in ids]
        q.put((rank, ids, gather_instance_stats(ids, stats, n, world)))
    finally:
        dist.destroy_process_group()


def test_batch_instance_sharding_two_gloo_ranks():
    """The batched form split by instance over two ranks: disjoint round-robin
    shards that cover every instance, and one all-gather that gives every rank
    all instances' stats in instance order (an instance's error status
    included)."""
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == [0, 2, 4, 6, 8, 10] and res[1][1] == [1, 3, 5, 7, 9]
    for _, _, full in res:
        assert [s["accepted"] for s in full] == [100 + i for i in range(11)]
        assert [s["status"] for s in full] == [-4 if i == 7 else 0 for i in range(11)]
        assert full[10]["t"] == pytest.approx(1e-10 + 10e-15)
    assert res[0][2] == res[1][2]
