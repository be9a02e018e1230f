"""Multi-process logic of bench.py on CPU (gloo, world size 2): every rank runs its own replica,
the job time is the maximum over ranks and the job throughput counts every rank's work."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.ranks_max(10.0 + 5.0 * rank)            # rank 1 is the slow one
    v = bench.job_throughput(4.0e9, 3, world, t)
    # the reference arm does its work on rank 0 only; other ranks return at once
    class A:
        steps, warmup, gpus = 1, 0, world
    r = bench.run_reference(A()) if rank == 1 else "skipped"
    out.put((rank, t, v, r))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_total_work():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, r in res:
        assert t == 15.0                                    # max over ranks
        assert abs(v - 4.0e9 * 3 * 2 / 15.0 / 1e9) < 1e-9   # both ranks' work over the slowest time
    assert res[1][3] is None                                # rank 1 did no reference work


def test_single_process_helpers():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ranks_max(3.5) == 3.5
    assert bench.job_throughput(1e9, 2, 1, 0.5) == 4.0
