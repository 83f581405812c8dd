"""Host logic of bench.py that needs no GPU: the max-over-ranks reduction of
the multi-rank run (two gloo ranks on CPU) and the seeded workloads."""
import os
import socket
import sys

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import bench
    d = bench.Dist(world)
    d.init("gloo")
    d.barrier()
    out[rank] = d.max(1.5 + rank)
    d.close()


def test_dist_max_over_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    ps = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in ps)
    assert out[0] == 2.5 and out[1] == 2.5


def test_bench_workloads_are_seeded():
    import bench
    a, b = bench.batched_problems(3), bench.batched_problems(3)
    for x, y in zip(a, b):
        assert np.array_equal(x["q0"], y["q0"]) and np.array_equal(x["target"], y["target"])
        assert 500 <= x["q0"].shape[0] <= 8000 and x["sigma"] in (0.05, 0.1, 0.2)
    tr = bench.served_trace(4)
    assert all(1000 <= r["q0"].shape[0] <= 50000 for r in tr)
    assert all(tr[k]["t_arrival"] < tr[k + 1]["t_arrival"] for k in range(3))
    q0, p0, t = bench.workload(64)
    assert q0.shape == (64, 3) and q0.dtype == np.float32 and np.array_equal(q0, bench.workload(64)[0])
