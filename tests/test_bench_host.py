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


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` times the FP64 oracle on the host cores and
    prints one JSON line with the reference arm's keys."""
    import json
    import subprocess
    root = os.path.dirname(HERE)
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--steps", "2",
                          "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "grad-evals/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1 and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "grad-evals/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["N"] == 4096 and d["config"]["T"] == 20
    # the same workload object the GPU arm reports: whole gradients, same config
    import bench
    assert d["config"] == bench.gshoot_config(4096, 1)
    assert "whole FP64 gradient" in d["cpu_baseline"]["sample"]


def test_clock_sampler_reads_median_under_load_and_reasons(tmp_path):
    """The clock record: median SM clock over the samples drawing at least the
    median power, the maximum clock, and every throttle reason seen active."""
    import subprocess
    import bench
    path = tmp_path / "clocks.csv"
    rows = [
        "1965, 2070, 150.0, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070, 450.0, Not Active, Not Active, Not Active, Not Active",
        "2070, 2070, 470.0, Not Active, Not Active, Not Active, Active",
        "2055, 2070, 460.0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    path.write_text("\n".join(rows) + "\n")
    s = bench.ClockSampler()
    s.path = str(path)
    s.proc = subprocess.Popen([sys.executable, "-c", "pass"])
    s.proc.wait()
    clk = s.stop()
    assert clk["samples"] == 4 and clk["sm_max_mhz"] == 2070.0
    assert clk["sm_mhz"] == 2062.5  # samples at or above the median draw (455 W): 2070 and 2055 MHz
    assert clk["reasons"] == ["sw_power_cap"] and clk["power_w_max"] == 470.0
    assert not os.path.exists(path)


def test_alu_peak_from_unit_counts():
    import bench
    assert abs(bench.alu_peak_tflops(152, 2070.0) - 80.54784) < 1e-9
