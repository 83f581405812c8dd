#!/usr/bin/env python
"""Benchmark of landmark geodesic shooting on GB300.

A step is one gradient evaluation: ComputeGradient of Algorithm 1.  It runs
the T forward Euler steps (StepForward pair sums plus the FP64 combine), the
loss of Eq. 3, then the T reverse steps (StepBackward pair sums plus the
adjoint combine), and assembles the gradient.  The workload is 4096 landmarks
on an ellipsoid with 8 Gaussian bumps for the target, sigma = 0.1,
lambda = 10, T = 20, and p0 ~ N(0, 0.01^2).  All inputs are synthetic and
seeded.

Metric: gradient evaluations per second.  Each step also reports its pair
interactions per second, 2 T N^2 / t.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gshoot|reference]

It prints one JSON line on rank 0.  `--impl reference` times the FP64 CPU
oracle on this host's cores on a bounded sample of the same workload.
Several GPUs run independent replicas.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import shutil
import subprocess
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

N_LANDMARKS = 4096
T_STEPS = 20
SIGMA = 0.1
LAMBDA = 10.0
P0_SCALE = 0.01
WORKLOAD = "ellipsoid landmarks N=4096 (8 bumps), sigma=0.1, lambda=10, T=20, p0~N(0,0.01^2)"
METRIC = "gradient evals/s (shoot_gradient, N=4096, T=20)"
# Algorithmic work per ordered landmark pair, counted from the formulas of
# StepForward / StepBackward (multiply, add and subtract = 1 flop, exp not
# counted).
FLOPS_PER_PAIR_FWD = 27
FLOPS_PER_PAIR_BWD = 65
# FP32 instructions per pair issued by the kernels (for the pipe fraction).
INSTR_PER_PAIR_FWD = 16
INSTR_PER_PAIR_BWD = 36


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gshoot", "reference"], default="gshoot")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--n", type=int, default=N_LANDMARKS,
                    help="landmark count (profiling runs only; the reported workload is N=4096)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def workload(n=N_LANDMARKS):
    import landmark_synth as ls
    pr = ls.ellipsoid_pair(n, seed=0, n_bumps=8)
    p0 = ls.random_momentum(n, P0_SCALE, seed=1)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return f(pr.q0), f(p0), f(pr.target)


# ---------------------------------------------------------------- distributed

class Dist:
    def __init__(self, gpus):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = False
        if self.world > 1:
            import torch.distributed as dist
            self.dist = dist

    def init(self, backend):
        if self.world > 1:
            self.dist.init_process_group(backend=backend)
            self.pg = True

    def barrier(self):
        if self.pg:
            self.dist.barrier()

    def max(self, x):
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.dist.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.dist.destroy_process_group()


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_uuid=None):
        self.proc = None
        self.path = None
        self.uuid = device_uuid

    def start(self):
        exe = shutil.which("nvidia-smi")
        if not exe:
            return
        import tempfile
        fd, self.path = tempfile.mkstemp(prefix="gs_clocks_", suffix=".csv")
        os.close(fd)
        cmd = [exe, "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.2)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 7:
                    rows.append(parts)
        os.unlink(self.path)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        sm, smax, power = [], [], []
        for r in rows:
            try:
                sm.append(float(r[0])); smax.append(float(r[1])); power.append(float(r[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if r[3 + k].lower().startswith("active"):
                    reasons.add(nm)
        # samples "under load": the upper half of the observed power draw
        if power:
            cut = np.median(power)
            loaded = [s for s, p in zip(sm, power) if p >= cut] or sm
        else:
            loaded = sm
        return {"sm_mhz": float(np.median(loaded)) if loaded else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": float(max(power)) if power else None}


# ---------------------------------------------------------------- peaks

def alu_peak_tflops(num_sms, max_mhz):
    # FP32 FMA pipe: 128 lanes per SM per clock, an FMA counts as 2 flops.
    return num_sms * 128 * 2 * max_mhz * 1e6 / 1e12


def read_measured_peaks():
    path = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


# ---------------------------------------------------------------- CPU oracle

def oracle_gradient_sample(min_seconds=10.0, max_evals=50):
    """Full FP64 oracle gradient evaluations of the workload, until ~min_seconds."""
    import oracle
    q0, p0, t = workload()
    q0, p0, t = (a.astype(np.float64) for a in (q0, p0, t))
    n_ev, t0 = 0, time.perf_counter()
    while True:
        oracle.shoot_gradient(q0, p0, t, T_STEPS, SIGMA, LAMBDA)
        n_ev += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or n_ev >= max_evals:
            break
    return {"value": n_ev / el, "unit": "grad-evals/s", "cores": oracle.max_threads(), "kind": "oracle",
            "sample": "%d full FP64 gradient evaluations of the workload (%.1f s)" % (n_ev, el)}


def run_reference(args, dist):
    """FP64 CPU oracle as the reference arm: each step is one time step of
    the workload (StepForward + StepBackward pair sums over all N^2 pairs),
    scaled to gradient evaluations (T such steps per evaluation)."""
    if dist.rank != 0:
        return 0
    import oracle
    q0, p0, t = workload()
    q = q0.astype(np.float64)
    p = p0.astype(np.float64)
    rng = np.random.default_rng(7)
    a = rng.normal(size=q.shape)
    b = rng.normal(size=q.shape)
    for _ in range(max(0, args.warmup)):
        oracle.step_forward(q, p, SIGMA)
        oracle.step_backward(q, p, a, b, SIGMA)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.step_forward(q, p, SIGMA)
        oracle.step_backward(q, p, a, b, SIGMA)
    el = time.perf_counter() - t0
    step_s = el / args.steps
    value = 1.0 / (T_STEPS * step_s)
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "grad-evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N_LANDMARKS, "T": T_STEPS, "sigma": SIGMA,
                   "lambda": LAMBDA, "step": "one time step (StepForward+StepBackward, all N^2 pairs)"},
        "cpu_baseline": {"value": value, "unit": "grad-evals/s", "cores": cores, "kind": "oracle",
                         "sample": "%d single time steps (fwd+bwd pair sums) scaled by T=%d" % (args.steps, T_STEPS)},
        "e2e": {"value": value, "unit": "grad-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "pair_interactions_per_s": 2 * N_LANDMARKS ** 2 / step_s,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm

def run_gshoot(args, dist):
    import torch
    import paper_1907_04839_gb300 as gsh

    dist.init("nccl")
    torch.cuda.set_device(dist.local)
    dev = torch.device("cuda", dist.local)
    lib = gsh.load()
    n = args.n
    q0, p0, t = workload(n)
    prm = gsh.GsParams(N=n, T=T_STEPS, ckpt_every=0, sigma=SIGMA, lambda_=LAMBDA,
                       lbfgs_m=10, max_iter=100, grad_tol=1e-5)
    dq, dp, dt = (torch.from_numpy(a).to(dev) for a in (q0, p0, t))
    gp = torch.empty((n, 3), dtype=torch.float32, device=dev)
    gq = torch.empty((n, 3), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sp = ctypes.c_void_p(stream.cuda_stream)
    P = lambda x: ctypes.c_void_p(x.data_ptr())

    def step_device():
        st = lib.shoot_gradient(ctypes.byref(prm), P(dq), P(dp), P(dt), None, P(gp), P(gq), sp)
        if st < 0:
            raise gsh.GShootError(st, lib.gs_last_error().decode())

    # correctness of the timed configuration against itself: finite loss
    loss = ctypes.c_double(0.0)
    gsh.check(lib.shoot_gradient(ctypes.byref(prm), P(dq), P(dp), P(dt), ctypes.byref(loss), P(gp), P(gq), sp))
    assert np.isfinite(loss.value)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)
    for _ in range(max(3, args.warmup)):
        step_device()
    torch.cuda.synchronize(dev)

    uuid = None
    try:
        u = torch.cuda.get_device_properties(dev).uuid
        uuid = "GPU-" + str(u) if u is not None and not str(u).startswith("GPU-") else str(u)
    except Exception:
        uuid = None
    clocks = ClockSampler(uuid)
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    for k in range(K):
        flush.fill_(float(k))          # untimed: evict L2 between steps
        ev[k][0].record(stream)
        step_device()
        ev[k][1].record(stream)
    torch.cuda.synchronize(dev)
    dist.barrier()
    clk = clocks.stop()
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms = dist.max(total_ms)
    ms_per_step = total_ms / K
    value = dist.world * K / (total_ms * 1e-3)

    # kernel times for the roofline (same kernels, same launch configuration)
    fwd_ms = ctypes.c_double(0.0)
    bwd_ms = ctypes.c_double(0.0)
    launches = ctypes.c_int32(0)
    gsh.check(lib.gs_time_pair_kernels(ctypes.byref(prm), P(dq), P(dp), P(dt), 200, ctypes.byref(fwd_ms),
                                       ctypes.byref(bwd_ms), ctypes.byref(launches), sp))

    # end to end: pinned host buffers through the C ABI, copies inside the timed region
    hq, hp, ht = (torch.from_numpy(a).pin_memory() for a in (q0, p0, t))
    hgp = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    hgq = torch.empty((n, 3), dtype=torch.float32).pin_memory()
    hl = ctypes.c_double(0.0)

    def step_host():
        st = lib.shoot_gradient(ctypes.byref(prm), P(hq), P(hp), P(ht), ctypes.byref(hl), P(hgp), P(hgq), sp)
        if st < 0:
            raise gsh.GShootError(st, lib.gs_last_error().decode())

    for _ in range(3):
        step_host()
    KE = max(1, min(args.e2e_steps, K))
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(KE):
        step_host()
    e2e_s = dist.max(time.perf_counter() - t0)
    e2e = {"value": dist.world * KE / e2e_s, "unit": "grad-evals/s",
           "h2d_bytes_per_step": 3 * n * 3 * 4, "d2h_bytes_per_step": 2 * n * 3 * 4 + 8,
           "steps": KE}

    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = read_measured_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    peak = alu_peak_tflops(num_sms, max_mhz)
    pairs = n * n
    bwd_tf = FLOPS_PER_PAIR_BWD * pairs / (bwd_ms.value * 1e-3) / 1e12
    fwd_tf = FLOPS_PER_PAIR_FWD * pairs / (fwd_ms.value * 1e-3) / 1e12
    pipe_lanes = num_sms * 128 * max_mhz * 1e6
    roofline = {
        "bound": "alu", "kernel": "k_step_backward (StepBackward pair sums + fused adjoint update)",
        "achieved": bwd_tf, "peak": peak, "unit": "TFLOP/s", "frac": bwd_tf / peak, "traffic": None,
        "peak_basis": "%d SMs x 128 FP32 lanes x 2 flops x %.0f MHz (max SM clock)" % (num_sms, max_mhz),
        "flops_per_launch": FLOPS_PER_PAIR_BWD * pairs, "launch_ms": bwd_ms.value,
        "fp32_pipe_frac": INSTR_PER_PAIR_BWD * pairs / (bwd_ms.value * 1e-3) / pipe_lanes,
        "forward": {"kernel": "k_step_forward", "achieved": fwd_tf, "frac": fwd_tf / peak,
                    "launch_ms": fwd_ms.value,
                    "fp32_pipe_frac": INSTR_PER_PAIR_FWD * pairs / (fwd_ms.value * 1e-3) / pipe_lanes},
    }
    line = {
        "metric": METRIC, "value": value, "unit": "grad-evals/s", "n_gpus": dist.world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if n == N_LANDMARKS else WORKLOAD.replace("N=4096", "N=%d" % n),
                   "N": n, "T": T_STEPS, "sigma": SIGMA, "lambda": LAMBDA,
                   "parallelism": "replicas" if dist.world > 1 else "single",
                   "l2": "flushed between steps (256 MiB write, untimed)",
                   "precision": "FP32 pair terms, compensated; double-single split combine; FP64 state/loss"},
        "pair_interactions_per_s": value * 2 * T_STEPS * pairs,
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": K * launches.value,
        "clocks": clk,
    }
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = oracle_gradient_sample()
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()
    return 0


def main():
    args = parse()
    dist = Dist(args.gpus)
    if args.impl == "reference":
        return run_reference(args, dist)
    return run_gshoot(args, dist)


if __name__ == "__main__":
    sys.exit(main())
