"""Multi-rank host logic of the benchmark on CPU ranks (gloo, world size 2).

The GPU path is replicas only: every rank solves its own right-hand sides and
the only collectives are the barrier and the max of the per-rank times.  Here
two gloo ranks check that reduction, the whole-job throughput it yields, that
the ranks' seeded inputs are disjoint, and that the reference arm runs on
rank 0 only.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from synthetic.sources import config_seed
    local = [1.5, 2.5][rank]
    mx = bench.max_over_ranks_of(local, dist, "cpu")
    val = bench.weak_scaling_value(local, 10, world, dist, "cpu")
    seeds = [config_seed(1, rank * 100 + i) for i in range(2)]
    gathered = [None] * world
    dist.all_gather_object(gathered, seeds)

    class A:
        steps, warmup = 1, 0
    ref_ran = bench.run_reference(A(), rank) if rank != 0 else "rank0"
    out[rank] = (mx, val, gathered, ref_ran)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_times_and_keep_inputs_disjoint():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(2):
        mx, val, gathered, ref = res[r]
        assert mx == 2.5
        assert val == pytest.approx(2 * 10 / 2.5)
        assert not set(gathered[0]) & set(gathered[1])
    assert res[1][3] is None  # rank 1 leaves the reference arm without work


def test_single_process_without_group():
    import bench
    assert bench.max_over_ranks_of(3.0) == 3.0
    assert bench.weak_scaling_value(2.0, 8, 1) == 4.0
