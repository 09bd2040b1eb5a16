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
