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
interactions per second, 2 T N^2 / t.  The same line carries two bounded
samples of the other workloads: `batched` (independent registrations packed
into shared launches, against a loop of single registrations), `served`
(a Poisson request trace through the continuous-batching server, with p50 /
p99 latency), `velocity` (the Eq. 4 velocity field on a 101^3 point grid and
points carried through the deformation), `population` (one template
registered to 34 subjects, with AverageDist / MaxDist) and `variants` (RK4
against Euler steps at equal pair work: speed and accuracy).
`--workload batched|served|population` runs one of those workloads at its
full size instead and prints its own line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gshoot|reference]
                    [--workload grad|batched|served|population]

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
# counted, factors common to all of a target's pairs applied once per target).
FLOPS_PER_PAIR_FWD = 27
FLOPS_PER_PAIR_BWD = 63
# FP32 instructions per pair issued by the kernels (for the pipe fraction).
INSTR_PER_PAIR_FWD = 16
INSTR_PER_PAIR_BWD = 36
# The velocity field of Eq. 4 per (point, landmark) pair: difference (3),
# squared distance (5), exponent scale (1), g p_j accumulated (6); issued
# FP32 lane-operations 9.
FLOPS_PER_PAIR_VEL = 15
INSTR_PER_PAIR_VEL = 9
# DRAM bytes (read + write) of one k_step_backward launch, from ncu
# (dram__bytes_read.sum + dram__bytes_write.sum, caches flushed before the
# launch) of the current kernel, by N.  Empty it whenever the kernel changes.
DRAM_BYTES_PER_BWD_LAUNCH = {4096: 425984}


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
    ap.add_argument("--workload", choices=["grad", "batched", "served", "population"], default="grad")
    ap.add_argument("--batched-count", type=int, default=None,
                    help="registrations of the batched workload (default: 128 in the grad run's sample, 512 alone)")
    ap.add_argument("--served-count", type=int, default=None,
                    help="requests of the served trace (default: 8 in the grad run's sample, 64 alone)")
    ap.add_argument("--no-samples", action="store_true",
                    help="grad run only (for profiling): no batched / served / other samples, no peak "
                         "microbenchmark (the roofline then uses the derived peak)")
    return ap.parse_args()


def workload(n=N_LANDMARKS):
    import landmark_synth as ls
    pr = ls.ellipsoid_pair(n, seed=0, n_bumps=8)
    p0 = ls.random_momentum(n, P0_SCALE, seed=1)
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return f(pr.q0), f(p0), f(pr.target)


def batched_problems(count):
    """Independent registrations: N log-uniform in [500, 8000], sigma uniform
    over {0.05, 0.1, 0.2}, lambda = 10, each its own ellipsoid-plus-bumps pair."""
    import landmark_synth as ls
    out = []
    for r in ls.batched_requests(count, n_lo=500, n_hi=8000, sigmas=(0.05, 0.1, 0.2), first_seed=1):
        pr = ls.ellipsoid_pair(r["n"], seed=r["seed"], n_bumps=8)
        out.append(dict(q0=np.ascontiguousarray(pr.q0, np.float32), target=np.ascontiguousarray(pr.target, np.float32),
                        sigma=r["sigma"], lam=LAMBDA))
    return out


def served_trace(count, rate=200.0):
    """Poisson arrivals (mean `rate` per second), N log-uniform in [1000, 50000],
    sigma = 0.1, lambda = 10."""
    import landmark_synth as ls
    out = []
    for r in ls.poisson_trace(count, rate, n_lo=1000, n_hi=50000, trace_seed=0, first_seed=1001):
        pr = ls.ellipsoid_pair(r["n"], seed=r["seed"], n_bumps=8)
        out.append(dict(q0=np.ascontiguousarray(pr.q0, np.float32), target=np.ascontiguousarray(pr.target, np.float32),
                        sigma=0.1, lam=LAMBDA, t_arrival=r["t_arrival"]))
    return out


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


def measure_peaks(lib, stream_ptr, uuid):
    """Measured throughput of the units the pair kernels run on
    (gs_measure_peaks: FFMA, paired FFMA2, MUFU ex2, FP64 DFMA chains on
    every SM, best of three ~50 ms launches, CUDA events), with the SM clock
    sampled while they run."""
    rates = (ctypes.c_double * 4)()
    kms = (ctypes.c_double * 4)()
    clocks = ClockSampler(uuid)
    clocks.start()
    st = lib.gs_measure_peaks(rates, kms, ctypes.c_double(50.0), stream_ptr)
    distinct = ctypes.c_double(0.0)
    st2 = lib.gs_measure_ffma2_distinct(ctypes.byref(distinct), ctypes.c_double(50.0), stream_ptr)
    clk = clocks.stop()
    if st != 0:
        return None
    return {"ffma_tflops": rates[0], "ffma2_tflops": rates[1], "fp32_tflops": max(rates[0], rates[1]),
            "ffma2_distinct_operands_tflops": distinct.value if st2 == 0 else None,
            "mufu_ex2_per_s": rates[2], "fp64_tflops": rates[3], "kernel_ms": [round(x, 3) for x in kms],
            "sm_mhz": clk.get("sm_mhz"), "clock_reasons": clk.get("reasons"),
            "basis": "gs_measure_peaks: 8 independent chains per thread, 4 x 256-thread CTAs per SM, "
                     "best of 3 launches of ~50 ms (CUDA events); ffma2_distinct_operands_tflops: the same "
                     "FFMA2 chains with three distinct register operands per instruction "
                     "(gs_measure_ffma2_distinct)"}


# ---------------------------------------------------------------- CPU oracle

def oracle_gradient_sample(min_seconds=10.0, max_evals=50):
    """The FP64 oracle on this host's cores, on bounded samples: whole
    gradient evaluations of the workload on all cores until ~min_seconds;
    one whole gradient on a single thread; and a whole registration of the
    smallest configuration (N = 256, T = 10, sigma = 0.2, 4 bumps, 50 L-BFGS
    iterations from p0 = 0) on all cores."""
    import oracle
    import landmark_synth as ls
    q0, p0, t = workload()
    q0, p0, t = (a.astype(np.float64) for a in (q0, p0, t))
    cores = oracle.max_threads()
    n_ev, t0 = 0, time.perf_counter()
    while True:
        oracle.shoot_gradient(q0, p0, t, T_STEPS, SIGMA, LAMBDA)
        n_ev += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or n_ev >= max_evals:
            break
    oracle.set_threads(1)
    try:
        t1 = time.perf_counter()
        oracle.shoot_gradient(q0, p0, t, T_STEPS, SIGMA, LAMBDA)
        el1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(cores)
    pr = ls.ellipsoid_pair(256, seed=0, n_bumps=4)
    rq, rt = (np.asarray(a, np.float32).astype(np.float64) for a in (pr.q0, pr.target))
    t2 = time.perf_counter()
    reg = oracle.register(rq, rt, 10, 0.2, LAMBDA, max_iter=50, grad_tol=0.0)
    el2 = time.perf_counter() - t2
    return {"value": n_ev / el, "unit": "grad-evals/s", "cores": cores, "kind": "oracle",
            "sample": "%d full FP64 gradient evaluations of the workload (%.1f s)" % (n_ev, el),
            "single_thread": {"value": 1.0 / el1, "unit": "grad-evals/s", "cores": 1,
                              "sample": "1 full FP64 gradient evaluation of the workload (%.1f s)" % el1},
            "register_n256": {"seconds": el2, "iters": reg["iters"], "evals": reg["evals"], "cores": cores,
                              "loss": reg["f"],
                              "sample": "oracle.register, N=256, T=10, sigma=0.2, lambda=10, 50 iterations"}}


def gshoot_config(n=N_LANDMARKS, world=1):
    """The `config` object both arms report for the gradient workload."""
    return {"workload": WORKLOAD if n == N_LANDMARKS else WORKLOAD.replace("N=4096", "N=%d" % n),
            "N": n, "T": T_STEPS, "sigma": SIGMA, "lambda": LAMBDA,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between steps (256 MiB write, untimed)",
            "precision": "FP32 pair terms, compensated; per-step split combine (see roofline.combine); "
                         "FP64 state/loss"}


def run_reference(args, dist):
    """FP64 CPU oracle as the reference arm: each step is one whole gradient
    evaluation of the workload (oracle.shoot_gradient: T forward steps, the
    loss, T reverse steps, all N^2 pairs each), on all host cores."""
    if dist.rank != 0:
        return 0
    import oracle
    q0, p0, t = workload()
    q, p, tt = (a.astype(np.float64) for a in (q0, p0, t))
    for _ in range(max(0, args.warmup)):
        oracle.shoot_gradient(q, p, tt, T_STEPS, SIGMA, LAMBDA)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.shoot_gradient(q, p, tt, T_STEPS, SIGMA, LAMBDA)
    el = time.perf_counter() - t0
    step_s = el / args.steps
    value = 1.0 / step_s
    cores = oracle.max_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "grad-evals/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": gshoot_config(N_LANDMARKS, 1),
        "cpu_baseline": {"value": value, "unit": "grad-evals/s", "cores": cores, "kind": "oracle",
                         "sample": "%d whole FP64 gradient evaluations of the workload (%.1f s)" % (args.steps, el)},
        "e2e": {"value": value, "unit": "grad-evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "pair_interactions_per_s": 2 * T_STEPS * N_LANDMARKS ** 2 / step_s,
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- batched and served workloads

def measure_batched(gsh, count, max_iter=100, T=T_STEPS):
    """`count` registrations two ways, each timed by wall clock from host
    inputs to host results: packed (register_batch: every time step of every
    resident problem in one launch) and a loop of register() calls."""
    import torch
    probs = batched_problems(count)
    gsh.register_batch(probs[:2], T=T, max_iter=2, grad_tol=1e-5)       # warm-up (module load)
    gsh.register(probs[0]["q0"], probs[0]["target"], T, probs[0]["sigma"], probs[0]["lam"], max_iter=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    packed = gsh.register_batch(probs, T=T, max_iter=max_iter, grad_tol=1e-5)
    torch.cuda.synchronize()
    t_packed = time.perf_counter() - t0
    t0 = time.perf_counter()
    loop = [gsh.register(p["q0"], p["target"], T, p["sigma"], p["lam"], max_iter=max_iter, grad_tol=1e-5)
            for p in probs]
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    pairs = lambda res: sum(2 * T * p["q0"].shape[0] ** 2 * r[1]["evals"] for p, r in zip(probs, res))
    rel = [abs(a[1]["loss"] - b[1]["loss"]) / max(abs(b[1]["loss"]), 1e-300) for a, b in zip(packed, loop)]
    ns = [p["q0"].shape[0] for p in probs]
    return {
        "registrations": count, "T": T, "max_iter": max_iter, "grad_tol": 1e-5,
        "N": "log-uniform [500, 8000], sum N^2 = %.3g" % float(sum(n * n for n in ns)),
        "packed_regs_per_s": count / t_packed, "loop_regs_per_s": count / t_loop,
        "speedup": t_loop / t_packed,
        "packed_pair_interactions_per_s": pairs(packed) / t_packed,
        "loop_pair_interactions_per_s": pairs(loop) / t_loop,
        "packed_s": t_packed, "loop_s": t_loop,
        "evals_packed": int(sum(r[1]["evals"] for r in packed)), "evals_loop": int(sum(r[1]["evals"] for r in loop)),
        "loss_rel_diff_median": float(np.median(rel)), "loss_rel_diff_max": float(np.max(rel)),
        "avg_dist_packed": float(np.mean([r[1]["avg_dist"] for r in packed])),
        "avg_dist_loop": float(np.mean([r[1]["avg_dist"] for r in loop])),
        "timing": "wall clock, host inputs and results included",
    }


def measure_served(gsh, count, max_iter=200, budget=120 << 30, rate=200.0, T=T_STEPS, schedule="fair"):
    """A Poisson trace through the continuous-batching server.  Requests are
    submitted at their arrival times while the server runs rounds; latency is
    from arrival to the round that finished the request.  schedule: the
    server's round schedule ("fair": equal pair work per request; "all":
    every resident request in every round; "lanes": small requests
    fair-scheduled in a second engine beside the all-rounds engine)."""
    trace = served_trace(count, rate)
    sv = gsh.Server(T=T, max_iter=max_iter, grad_tol=1e-5, memory_budget=budget, max_problems=1024,
                    schedule=schedule)
    rid = [None] * count
    done_at = [None] * count
    service = [None] * count
    evals = [0] * count
    infos = [None] * count
    t0 = time.perf_counter()
    nsub = 0
    outstanding = set()
    while True:
        now = time.perf_counter() - t0
        while nsub < count and trace[nsub]["t_arrival"] <= now:
            r = trace[nsub]
            rid[nsub] = sv.submit(r["q0"], r["target"], r["sigma"], r["lam"])
            outstanding.add(nsub)
            nsub += 1
        if not outstanding:
            if nsub == count:
                break
            time.sleep(max(0.0, trace[nsub]["t_arrival"] - (time.perf_counter() - t0)))
            continue
        a, q, c = sv.step()
        if c > 0:
            tw = time.perf_counter() - t0
            for k in list(outstanding):
                out = sv.poll(rid[k])
                if out is not None:
                    done_at[k] = tw
                    service[k] = out[2][1]
                    evals[k] = out[1]["evals"]
                    infos[k] = out[1]
                    outstanding.discard(k)
    sv.close()
    lat = np.array([done_at[k] - trace[k]["t_arrival"] for k in range(count)])
    svc = np.array(service)
    makespan = max(done_at) - trace[0]["t_arrival"]
    ns = [r["q0"].shape[0] for r in trace]
    return {
        "requests": count, "schedule": schedule, "arrival_rate_per_s": rate, "T": T, "max_iter": max_iter,
        "grad_tol": 1e-5,
        "memory_budget_bytes": budget, "N": "log-uniform [1000, 50000], mean %.0f" % float(np.mean(ns)),
        "regs_per_s": count / makespan, "makespan_s": makespan,
        "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
        "service_p50_s": float(np.percentile(svc, 50)), "service_p99_s": float(np.percentile(svc, 99)),
        "pair_interactions_per_s": sum(2 * T * n * n * e for n, e in zip(ns, evals)) / makespan,
        "timing": "wall clock from arrival to result, host inputs, queueing included",
        "per_request": [{"N": ns[k], "iters": infos[k]["iters"], "evals": infos[k]["evals"],
                         "status": infos[k]["status"], "loss": infos[k]["loss"],
                         "grad_ratio": infos[k]["grad_norm"] / max(infos[k]["grad_norm0"], 1e-300),
                         "avg_dist": infos[k]["avg_dist"], "max_dist": infos[k]["max_dist"],
                         "latency_s": float(lat[k]), "service_s": float(svc[k]),
                         "queue_s": float(lat[k] - svc[k])} for k in range(count)],
    }


def measure_population(gsh, subjects=34, n=1847, T=40, max_iter=400, sigma=SIGMA, lam=LAMBDA):
    """One template registered to every subject of a population (the shape
    of the paper's study: 34 subjects, 1847 landmarks, T = 40, at most 400
    iterations), packed into one register_batch call and, for comparison,
    as a loop of register() calls.  Wall clock, host inputs and results
    included.  Reports AverageDist / MaxDist (Section 3.1) before and after,
    mean and standard deviation over the subjects, as in Table 1."""
    import torch
    import landmark_synth as ls
    pop = ls.population(n, subjects, seed=0)
    q0 = np.ascontiguousarray(pop.template, np.float32)
    probs = [dict(q0=q0, target=np.ascontiguousarray(t, np.float32), sigma=sigma, lam=lam) for t in pop.targets]
    gsh.register_batch(probs[:2], T=T, max_iter=2, grad_tol=1e-5)       # warm-up
    gsh.register(q0, probs[0]["target"], T, sigma, lam, max_iter=2)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    packed = gsh.register_batch(probs, T=T, max_iter=max_iter, grad_tol=1e-5)
    torch.cuda.synchronize()
    t_packed = time.perf_counter() - t0
    t0 = time.perf_counter()
    loop = [gsh.register(q0, p["target"], T, sigma, lam, max_iter=max_iter, grad_tol=1e-5) for p in probs]
    torch.cuda.synchronize()
    t_loop = time.perf_counter() - t0
    before = [np.linalg.norm(p["target"].astype(np.float64) - q0.astype(np.float64), axis=1) for p in probs]
    ms = lambda xs: [float(np.mean(xs)), float(np.std(xs))]
    evals = int(sum(r[1]["evals"] for r in packed))
    return {
        "subjects": subjects, "N": n, "T": T, "sigma": sigma, "lambda": lam, "max_iter": max_iter,
        "grad_tol": 1e-5, "template": "mean of the subjects (synthetic population, seed 0)",
        "packed_regs_per_s": subjects / t_packed, "loop_regs_per_s": subjects / t_loop,
        "speedup": t_loop / t_packed, "packed_s": t_packed, "loop_s": t_loop,
        "packed_pair_interactions_per_s": 2.0 * T * n * n * evals / t_packed,
        "evals_packed": evals, "evals_loop": int(sum(r[1]["evals"] for r in loop)),
        "iters_mean": float(np.mean([r[1]["iters"] for r in packed])),
        "avg_dist_before": ms([b.mean() for b in before]), "max_dist_before": ms([b.max() for b in before]),
        "avg_dist_after": ms([r[1]["avg_dist"] for r in packed]),
        "max_dist_after": ms([r[1]["max_dist"] for r in packed]),
        "avg_dist_after_loop": ms([r[1]["avg_dist"] for r in loop]),
        "dist_basis": "[mean, std] over subjects of AverageDist / MaxDist(q(1), target)",
        "timing": "wall clock, host inputs and results included",
    }


def planar_rate(gsh, reps):
    """Gradient evaluations per second for planar landmarks: 4096 points on
    an ellipse with semi-axes 1.0 / 0.6 (8 bumps), sigma = 0.05, T = 20,
    lambda = 10; device inputs, CUDA events.  The momenta are the smooth
    field (target - q0) / (kernel row mass), about sqrt(2 pi) sigma N /
    perimeter."""
    import math
    import torch
    import landmark_synth as ls
    dev = torch.device("cuda", torch.cuda.current_device())
    pr = ls.ellipse_pair(N_LANDMARKS, seed=0, n_bumps=8)
    mass = math.sqrt(2 * math.pi) * 0.05 * N_LANDMARKS / (2 * math.pi * math.sqrt((1.0 + 0.36) / 2))
    p0 = (pr.target - pr.q0) / mass
    dq, dp, dt = (torch.tensor(np.asarray(a, np.float32), device=dev) for a in (pr.q0, p0, pr.target))
    stream = torch.cuda.current_stream(dev)
    f = lambda: gsh.shoot_gradient(dq, dp, dt, T_STEPS, 0.05, LAMBDA)
    for _ in range(3):
        f()
    torch.cuda.synchronize(dev)
    out = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        f()
        b.record(stream)
        b.synchronize()
        out.append(a.elapsed_time(b))
    ms = float(np.median(out))
    return {"N": N_LANDMARKS, "T": T_STEPS, "sigma": 0.05, "grad_evals_per_s": 1e3 / ms,
            "pair_interactions_per_s": 2 * T_STEPS * N_LANDMARKS ** 2 / (ms * 1e-3)}


def measure_variants(gsh, reps=50, fit_iters=30):
    """The RK4 integrator against the paper's Euler steps at equal pair work
    (RK4 with T = 5 evaluates the pair sums 20 times per sweep, as Euler
    with T = 20 does): gradient evaluations per second of each (device
    inputs, CUDA events, median of `reps`), and the error of each q(1)
    against an RK4 solution with T = 80, relative to the displacement
    q(1) - q0.  The momenta are those of a registration of the workload
    (`fit_iters` L-BFGS iterations from zero), so the flow is the smooth
    deformation a registration produces."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    q0, _, t = workload()
    p0, _ = gsh.register(q0, t, T_STEPS, SIGMA, LAMBDA, max_iter=fit_iters, grad_tol=0.0)
    p0 = np.ascontiguousarray(p0, np.float32)
    dq, dp, dt = (torch.from_numpy(a).to(dev) for a in (q0, p0, t))
    stream = torch.cuda.current_stream(dev)

    def rate(T, integ, h_at="start"):
        f = lambda: gsh.shoot_gradient(dq, dp, dt, T, SIGMA, LAMBDA, integrator=integ, h_at=h_at)
        for _ in range(3):
            f()
        torch.cuda.synchronize(dev)
        out = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            f()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return 1e3 / float(np.median(out))

    ref = gsh.shoot_forward(dq, dp, 80, SIGMA, integrator="rk4")[0].double()
    disp = float(torch.linalg.norm(ref - dq.double()))
    err = lambda T, integ: float(torch.linalg.norm(gsh.shoot_forward(dq, dp, T, SIGMA, integrator=integ)[0].double()
                                                   - ref)) / disp
    return {
        "N": q0.shape[0], "p0": "%d L-BFGS iterations of the workload's registration" % fit_iters,
        "reference": "RK4, T = 80", "displacement_rms": disp / np.sqrt(q0.shape[0]),
        "euler_T20": {"grad_evals_per_s": rate(20, "euler"), "q1_rel_err": err(20, "euler")},
        "rk4_T5": {"grad_evals_per_s": rate(5, "rk4"), "q1_rel_err": err(5, "rk4")},
        "rk4_T5_kinetic_end": {"grad_evals_per_s": rate(5, "rk4", "end")},
        "planar_euler_T20": planar_rate(gsh, reps),
        "timing": "shoot_gradient through the binding, CUDA events, median of %d" % reps,
    }


def velocity_grid(n_side=101, half=1.2):
    """Query points of the deformation: a regular n_side^3 grid over the
    box [-half, half]^3 that holds the ellipsoid (an image grid stand-in)."""
    ax = np.linspace(-half, half, n_side, dtype=np.float64)
    g = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    return np.ascontiguousarray(g, dtype=np.float32)


def measure_velocity(gsh, reps=5, T=T_STEPS, peak=None):
    """The Eq. 4 velocity field: a 101^3 grid of points carried through the
    deformation of the workload's landmarks (flow_points: the landmark flow
    plus T Euler steps of every point), and one velocity_field evaluation at
    the same points.  Device-resident inputs, CUDA events on the stream,
    median of `reps` calls after one warm-up."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    q0, p0, _ = workload()
    x = velocity_grid()
    n, m = q0.shape[0], x.shape[0]
    dq, dp, dx = (torch.from_numpy(a).to(dev) for a in (q0, p0, x))
    stream = torch.cuda.current_stream(dev)

    def timed(fn):
        fn()
        torch.cuda.synchronize(dev)
        out = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            out.append(a.elapsed_time(b))
        return float(np.median(out))

    t_flow = timed(lambda: gsh.flow_points(dq, dp, dx, T, SIGMA))
    t_vel = timed(lambda: gsh.velocity_field(dq, dp, dx, SIGMA))
    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if peak is None:
        peak = alu_peak_tflops(num_sms, float(read_measured_peaks().get("sm_max_mhz", 2070.0)))
    pairs_vel = float(m) * n
    tf = FLOPS_PER_PAIR_VEL * pairs_vel / (t_vel * 1e-3) / 1e12
    return {
        "N": n, "M": m, "T": T, "points": "regular 101^3 grid over [-1.2, 1.2]^3",
        "flow_points_ms": t_flow, "point_steps_per_s": m * T / (t_flow * 1e-3),
        "flow_pair_interactions_per_s": T * pairs_vel / (t_flow * 1e-3),
        "velocity_field_ms": t_vel, "velocity_pair_interactions_per_s": pairs_vel / (t_vel * 1e-3),
        "roofline": {"bound": "alu", "kernel": "k_velocity (one velocity_field call, conversions included)",
                     "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                     "fp32_pipe_frac": INSTR_PER_PAIR_VEL * pairs_vel / (t_vel * 1e-3) / (peak * 1e12 / 2)},
        "timing": "CUDA events on the stream, device inputs, median of %d calls" % reps,
    }


def _grad_inputs(dev, n, sigma_seed=0):
    import torch
    import landmark_synth as ls
    pr = ls.ellipsoid_pair(n, seed=sigma_seed, n_bumps=8)
    p0 = ls.random_momentum(n, P0_SCALE, seed=sigma_seed + 1)
    return tuple(torch.tensor(np.asarray(a, np.float32), device=dev) for a in (pr.q0, p0, pr.target))


def _timed_gradients(lib, prm, bufs, stream, reps, flush):
    """Median device time (ms) of one shoot_gradient call and of its forward
    and reverse sweeps (phase events), L2 flushed before each call."""
    import torch
    P = lambda x: ctypes.c_void_p(x.data_ptr())
    q, p, t, gp, gq = bufs
    sp = ctypes.c_void_p(stream.cuda_stream)
    call = lambda: lib.shoot_gradient(ctypes.byref(prm), P(q), P(p), P(t), None, P(gp), P(gq), sp)
    import paper_1907_04839_gb300 as gsh
    gsh.check(lib.gs_set_phase_timing(1))
    try:
        for _ in range(3):
            gsh.check(call())
        tt, fw, bw = [], [], []
        pf, pb = ctypes.c_double(0.0), ctypes.c_double(0.0)
        for r in range(reps):
            flush.fill_(float(r))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gsh.check(call())
            b.record(stream)
            b.synchronize()
            tt.append(a.elapsed_time(b))
            gsh.check(lib.gs_phase_times(ctypes.byref(pf), ctypes.byref(pb)))
            fw.append(pf.value)
            bw.append(pb.value)
    finally:
        gsh.check(lib.gs_set_phase_timing(0))
    return float(np.median(tt)), float(np.median(fw)), float(np.median(bw))


def roofline_at(gsh, lib, dev, n, peak, mufu_peak, T=T_STEPS, sigma=0.05, reps=8):
    """The step kernels' roofline at a larger N (16384 landmarks: several
    waves per launch, where the pair loops rather than the fixed per-launch
    costs set the time): whole gradients of an ellipsoid workload
    (sigma = 0.05, T = 20), per-launch times from the graph's phase events
    (sweep / T)."""
    import torch
    q, p, t = _grad_inputs(dev, n)
    bufs = (q, p, t, torch.empty_like(q), torch.empty_like(q))
    prm = gsh.GsParams(N=n, T=T, ckpt_every=0, sigma=sigma, lambda_=LAMBDA, lbfgs_m=10, max_iter=1, grad_tol=0.0)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    ms, fwd, bwd = _timed_gradients(lib, prm, bufs, torch.cuda.current_stream(dev), reps, flush)
    del flush
    pairs = float(n) * n
    lanes = peak * 1e12 / 2
    out = {"N": n, "T": T, "sigma": sigma, "gradient_ms": ms, "peak": peak, "unit": "TFLOP/s",
           "basis": "per-launch time = sweep time / T from graph events, median of %d gradients" % reps}
    for name, sweep, fl, ins, kind in (("reverse", bwd, FLOPS_PER_PAIR_BWD, INSTR_PER_PAIR_BWD, 1),
                                       ("forward", fwd, FLOPS_PER_PAIR_FWD, INSTR_PER_PAIR_FWD, 0)):
        launch = sweep / T * 1e-3
        th, cl = ctypes.c_int32(0), ctypes.c_int32(0)
        gsh.check(lib.gs_step_config(kind, n, 0, 0, ctypes.byref(th), ctypes.byref(cl)))
        out[name] = {"launch_ms": launch * 1e3, "achieved": fl * pairs / launch / 1e12,
                     "frac": fl * pairs / launch / 1e12 / peak, "fp32_pipe_frac": ins * pairs / launch / lanes,
                     "xu_frac": pairs / launch / mufu_peak, "launch_shape": {"threads": th.value, "cluster": cl.value}}
    return out


def measure_combine(gsh, lib, dev, sizes=(4096, 16384)):
    """Whole gradients with the split partials of each step added in
    double-single arithmetic and in FP64 (gs_set_combine_precision), same
    inputs, same process."""
    import torch
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out = {"basis": "median device time of whole gradients (T=20, sigma=0.1), L2 flushed"}
    cur = None
    try:
        for n in sizes:
            q, p, t = _grad_inputs(dev, n)
            bufs = (q, p, t, torch.empty_like(q), torch.empty_like(q))
            prm = gsh.GsParams(N=n, T=T_STEPS, ckpt_every=0, sigma=SIGMA, lambda_=LAMBDA, lbfgs_m=10, max_iter=1,
                               grad_tol=0.0)
            row = {}
            for f64 in (0, 1):
                gsh.check(lib.gs_set_combine_precision(f64))
                ms, fw, bw = _timed_gradients(lib, prm, bufs, torch.cuda.current_stream(dev),
                                              20 if n <= 4096 else 6, flush)
                row["fp64" if f64 else "double_single"] = {"gradient_ms": ms, "forward_ms": fw, "reverse_ms": bw}
            row["fp64_extra_pct"] = 100.0 * (row["fp64"]["gradient_ms"] / row["double_single"]["gradient_ms"] - 1)
            out["N%d" % n] = row
    finally:
        gsh.check(lib.gs_set_combine_precision(0))
    del flush
    return out


def measure_register_small(gsh):
    """A whole registration of the smallest configuration (N = 256, T = 10,
    sigma = 0.2, lambda = 10, 4 bumps, 50 L-BFGS iterations from p0 = 0),
    host arrays in and out, wall clock (median of 3)."""
    import landmark_synth as ls
    pr = ls.ellipsoid_pair(256, seed=0, n_bumps=4)
    q0, t = (np.ascontiguousarray(a, np.float32) for a in (pr.q0, pr.target))
    gsh.register(q0, t, 10, 0.2, LAMBDA, max_iter=5, grad_tol=0.0)
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        _, info = gsh.register(q0, t, 10, 0.2, LAMBDA, max_iter=50, grad_tol=0.0)
        ts.append(time.perf_counter() - t0)
    return {"seconds": float(np.median(ts)), "iters": info["iters"], "evals": info["evals"], "loss": info["loss"],
            "timing": "register() wall clock, host arrays, median of 3"}


def measure_served_vs_plain(gsh, count, max_iter=200, T=T_STEPS):
    """The served workload five ways, on the same first `count` requests of
    the trace: (1) the server with two lanes (schedule "lanes": requests of
    at most 8192 landmarks fair-scheduled in a second engine, on a stream of
    the highest priority, beside the all-rounds rounds of the larger ones)
    under the trace's 200/s arrivals (overload: its completion rate is the
    capacity); (2) the same with every resident request in every round
    (schedule "all": the most packing, no latency advantage for small
    requests); (2b) the fair schedule alone (equal pair work per request);
    (3) the server of (1) under a Poisson rate of half its capacity, so that
    latency percentiles describe a stable queue; (4) the plain
    single-registration path, one register() call after another in arrival
    order, each timed, with the latencies a single plain worker would give
    under the same arrival processes.  Accuracy of (1) against (4):
    per-request final loss, AverageDist and MaxDist."""
    import landmark_synth as ls
    burst = measure_served(gsh, count, max_iter=max_iter, T=T, schedule="lanes")
    every = measure_served(gsh, count, max_iter=max_iter, T=T, schedule="all")
    fair = measure_served(gsh, count, max_iter=max_iter, T=T, schedule="fair")
    cap = burst["regs_per_s"]
    sub = measure_served(gsh, count, max_iter=max_iter, T=T, rate=0.5 * cap, schedule="lanes")
    trace = served_trace(count)
    svc, infos = [], []
    for r in trace:
        t0 = time.perf_counter()
        _, info = gsh.register(r["q0"], r["target"], T, r["sigma"], r["lam"], max_iter=max_iter, grad_tol=1e-5)
        svc.append(time.perf_counter() - t0)
        infos.append(info)

    def fifo(arrivals):
        end, lat = 0.0, []
        for a, s in zip(arrivals, svc):
            end = max(end, a) + s
            lat.append(end - a)
        return np.array(lat), end - arrivals[0]

    arr_burst = [r["t_arrival"] for r in trace]
    arr_sub = [r["t_arrival"] for r in ls.poisson_trace(count, 0.5 * cap, n_lo=1000, n_hi=50000, trace_seed=0,
                                                        first_seed=1001)]
    lat_b, mk_b = fifo(arr_burst)
    lat_s, mk_s = fifo(arr_sub)
    served_loss = [q["loss"] for q in burst["per_request"]]
    rel = [abs(a - b["loss"]) / max(abs(b["loss"]), 1e-300) for a, b in zip(served_loss, infos)]
    plain = {
        "regs_per_s": count / float(np.sum(svc)), "service_s": [round(x, 3) for x in svc],
        "latency_p50_s_at_200_per_s": float(np.percentile(lat_b, 50)),
        "latency_p99_s_at_200_per_s": float(np.percentile(lat_b, 99)),
        "latency_p50_s_at_half_capacity": float(np.percentile(lat_s, 50)),
        "latency_p99_s_at_half_capacity": float(np.percentile(lat_s, 99)),
        "makespan_s_at_200_per_s": mk_b,
        "avg_dist_mean": float(np.mean([i["avg_dist"] for i in infos])),
        "max_dist_mean": float(np.mean([i["max_dist"] for i in infos])),
        "status": [int(i["status"]) for i in infos],
        "timing": "register() wall clock per request, host arrays; latencies of one FIFO worker",
    }
    burst["capacity_regs_per_s"] = cap
    burst["half_capacity"] = {k: sub[k] for k in ("arrival_rate_per_s", "regs_per_s", "makespan_s", "latency_p50_s",
                                                 "latency_p99_s", "service_p50_s", "service_p99_s")}
    burst["plain_loop"] = plain
    burst["served_over_plain_regs_per_s"] = burst["regs_per_s"] / plain["regs_per_s"]
    burst["schedule_all"] = {k: every[k] for k in ("regs_per_s", "makespan_s", "latency_p50_s", "latency_p99_s",
                                                  "service_p50_s", "service_p99_s", "pair_interactions_per_s")}
    burst["schedule_all"]["served_over_plain_regs_per_s"] = every["regs_per_s"] / plain["regs_per_s"]
    burst["lane_split"] = 8192
    burst["schedule_fair"] = {k: fair[k] for k in ("regs_per_s", "makespan_s", "latency_p50_s", "latency_p99_s",
                                                  "service_p50_s", "service_p99_s", "pair_interactions_per_s")}
    burst["schedule_fair"]["served_over_plain_regs_per_s"] = fair["regs_per_s"] / plain["regs_per_s"]
    burst["accuracy_vs_plain"] = {
        "loss_rel_diff_median": float(np.median(rel)), "loss_rel_diff_max": float(np.max(rel)),
        "avg_dist_mean_served": float(np.mean([q["avg_dist"] for q in burst["per_request"]])),
        "max_dist_mean_served": float(np.mean([q["max_dist"] for q in burst["per_request"]]))}
    return burst


def run_workload(args, dist):
    """--workload batched|served: the full-size workload, its own JSON line."""
    import torch
    import paper_1907_04839_gb300 as gsh
    dist.init("nccl")
    torch.cuda.set_device(dist.local)
    if args.workload == "batched":
        res = measure_batched(gsh, args.batched_count or 512)
        metric = "registrations/s (%d packed registrations, N~LogU[500,8000], T=20)" % res["registrations"]
        value, ms = res["packed_regs_per_s"], res["packed_s"] * 1e3
    elif args.workload == "population":
        res = measure_population(gsh)
        metric = "registrations/s (one template to 34 subjects, N=1847, T=40, packed)"
        value, ms = res["packed_regs_per_s"], res["packed_s"] * 1e3
    else:
        res = measure_served_vs_plain(gsh, args.served_count or 64)
        metric = "served registrations/s (Poisson 200/s, N~LogU[1000,50000], T=20)"
        value, ms = res["regs_per_s"], res["makespan_s"] * 1e3
    line = {"metric": metric, "value": value * dist.world, "unit": "regs/s", "n_gpus": dist.world, "steps": 1,
            "warmup": 1, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": {"workload": args.workload, **res}}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)
    dist.close()
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
    # (--no-samples, the profiling command, runs the gradient's kernels only)
    peaks_meas = None if args.no_samples else measure_peaks(lib, sp, uuid)
    clocks = ClockSampler(uuid)
    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    # The graph records events around its forward and reverse sweeps: the
    # per-launch times of the roofline come from the timed steps themselves.
    gsh.check(lib.gs_set_phase_timing(1))
    step_device()
    torch.cuda.synchronize(dev)
    fwd_phase = bwd_phase = 0.0
    pf, pb = ctypes.c_double(0.0), ctypes.c_double(0.0)
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.start()
    for k in range(K):
        flush.fill_(float(k))          # untimed: evict L2 between steps
        ev[k][0].record(stream)
        step_device()
        ev[k][1].record(stream)
        ev[k][1].synchronize()         # host-side wait, outside the events
        gsh.check(lib.gs_phase_times(ctypes.byref(pf), ctypes.byref(pb)))
        fwd_phase += pf.value
        bwd_phase += pb.value
    torch.cuda.synchronize(dev)
    dist.barrier()
    clk = clocks.stop()
    gsh.check(lib.gs_set_phase_timing(0))
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
    # three blocks of KE / 3 calls; the median block is reported
    nb = 3 if KE >= 3 else 1
    per = KE // nb
    rates = []
    for _ in range(nb):
        dist.barrier()
        t0 = time.perf_counter()
        for _ in range(per):
            step_host()
        rates.append(dist.world * per / dist.max(time.perf_counter() - t0))
    e2e = {"value": float(np.median(rates)), "unit": "grad-evals/s",
           "h2d_bytes_per_step": 3 * n * 3 * 4, "d2h_bytes_per_step": 2 * n * 3 * 4 + 8,
           "steps": per * nb, "blocks": [round(r, 1) for r in rates],
           "path": "shoot_gradient with pinned host q0, p0, target in and grad_p0, grad_q0, loss out"}

    num_sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = read_measured_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    derived_peak = alu_peak_tflops(num_sms, max_mhz)
    if peaks_meas:
        peak = peaks_meas["ffma2_tflops"]
        peak_basis = ("measured: paired FP32 FFMA2 chains on all %d SMs (gs_measure_peaks), %.1f TFLOP/s at a "
                      "median %s MHz; derived %d x 128 lanes x 2 x %.0f MHz = %.1f TFLOP/s" % (
                          num_sms, peak, peaks_meas.get("sm_mhz"), num_sms, max_mhz, derived_peak))
        mufu_peak = peaks_meas["mufu_ex2_per_s"]
    else:
        peak = derived_peak
        peak_basis = "%d SMs x 128 FP32 lanes x 2 flops x %.0f MHz (derived: not measured in this run)" % (
            num_sms, max_mhz)
        mufu_peak = num_sms * 32 * max_mhz * 1e6
    pairs = n * n
    # average launch duration in the timed steps: sweep time / T launches
    bwd_launch_ms = bwd_phase / (K * T_STEPS)
    fwd_launch_ms = fwd_phase / (K * T_STEPS)
    bwd_tf = FLOPS_PER_PAIR_BWD * pairs / (bwd_launch_ms * 1e-3) / 1e12
    fwd_tf = FLOPS_PER_PAIR_FWD * pairs / (fwd_launch_ms * 1e-3) / 1e12
    pipe_lanes = peak * 1e12 / 2  # FP32 lane-operations per second at the measured rate
    traffic = DRAM_BYTES_PER_BWD_LAUNCH.get(n)
    shape = {}
    for kind, name in ((0, "forward"), (1, "reverse")):
        t, c = ctypes.c_int32(0), ctypes.c_int32(0)
        gsh.check(lib.gs_step_config(kind, n, 0, 0, ctypes.byref(t), ctypes.byref(c)))
        shape[name] = {"threads": t.value, "cluster": c.value}
    roofline = {
        "bound": "alu", "kernel": "k_step_backward (StepBackward pair sums + fused adjoint update)",
        "achieved": bwd_tf, "peak": peak, "unit": "TFLOP/s", "frac": bwd_tf / peak, "traffic": traffic,
        "peak_basis": peak_basis,
        "flops_per_launch": FLOPS_PER_PAIR_BWD * pairs, "launch_ms": bwd_launch_ms,
        "launch_ms_basis": "reverse-sweep time / T from graph events in the timed steps (gaps included)",
        "isolated_launch_ms": bwd_ms.value,
        "launch_shape": shape["reverse"],
        "fp32_pipe_frac": INSTR_PER_PAIR_BWD * pairs / (bwd_launch_ms * 1e-3) / pipe_lanes,
        "xu_frac": pairs / (bwd_launch_ms * 1e-3) / mufu_peak,
        "forward": {"kernel": "k_step_forward", "achieved": fwd_tf, "frac": fwd_tf / peak,
                    "launch_ms": fwd_launch_ms, "isolated_launch_ms": fwd_ms.value,
                    "launch_shape": shape["forward"],
                    "fp32_pipe_frac": INSTR_PER_PAIR_FWD * pairs / (fwd_launch_ms * 1e-3) / pipe_lanes,
                    "xu_frac": pairs / (fwd_launch_ms * 1e-3) / mufu_peak},
        "peaks": peaks_meas,
        "combine": None if args.no_samples else measure_combine(gsh, lib, dev),
    }
    distinct = (peaks_meas or {}).get("ffma2_distinct_operands_tflops")
    if distinct:
        # the same lane-operation rates against FFMA2 with three distinct register operands
        roofline["fp32_pipe_frac_vs_distinct_operand_ffma2"] = roofline["fp32_pipe_frac"] * peak / distinct
        roofline["forward"]["fp32_pipe_frac_vs_distinct_operand_ffma2"] = (
            roofline["forward"]["fp32_pipe_frac"] * peak / distinct)
    roofline_large = None if args.no_samples else roofline_at(gsh, lib, dev, 16384, peak, mufu_peak)
    line = {
        "metric": METRIC, "value": value, "unit": "grad-evals/s", "n_gpus": dist.world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": gshoot_config(n, dist.world),
        "pair_interactions_per_s": value * 2 * T_STEPS * pairs,
        "roofline": roofline,
        "roofline_n16384": roofline_large,
        "e2e": e2e,
        "gpu_launches": K * launches.value,
        "clocks": clk,
    }
    if not args.no_samples:
        line["register_n256"] = measure_register_small(gsh)
        line["batched"] = measure_batched(gsh, args.batched_count or 128)
        line["served"] = measure_served_vs_plain(gsh, args.served_count or 8)
        line["velocity"] = measure_velocity(gsh, peak=peak)
        line["population"] = measure_population(gsh)
        line["variants"] = measure_variants(gsh)
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
    if args.workload != "grad":
        return run_workload(args, dist)
    return run_gshoot(args, dist)


if __name__ == "__main__":
    sys.exit(main())
