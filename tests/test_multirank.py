"""The N > 1 path of bench.py on CPU with two gloo ranks: the slowest
rank's time is taken by an all-reduce MAX, the whole-job throughput counts
the steps of every rank, and under torchrun only rank 0 runs the oracle's
reference arm (the other ranks return at once)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0, 12.5][rank]
    ms = bench.slowest_rank_ms(local, world, "cpu")
    torch.distributed.barrier()
    ref = bench.run_reference(None, rank, world) if rank != 0 else "skipped"
    q.put((rank, ms, bench.job_throughput(ms, 5, world), ref))
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[1] for o in out] == [12.5, 12.5]            # the slowest rank's time
    assert all(abs(o[2] - 2 * 5 / 12.5e-3) < 1e-9 for o in out)   # 800 steps/s
    assert out[1][3] is None                              # rank 1: no reference work
