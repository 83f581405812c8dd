"""Sweep the pair-sum kernel variants and split counts on the current GPU.

    python -m paper_1907_04839_gb300.tune [--n 4096 16384] [--reps 50]

For each landmark count N, the sweep times every (threads per CTA, targets
per thread) variant of StepForward and StepBackward.  Each variant is tried
at the library's balanced split count and at split counts that place a whole
number of CTAs on every SM.  Timing goes through gs_time_pair_config.  The
output is one JSON line per measurement.  Inputs are seeded ellipsoid
landmarks.

`--policy 0 1 2` repeats the fused-kernel sweep under each cluster
scheduling preference (default, spread, load balancing) and reports how many
clusters of each shape can be resident at once; `--graph` times the fused
kernels as back-to-back replays inside a CUDA graph.

`--emit-table PATH` measures the step-configuration table the library
compiles in (csrc/step_table.inc).  For every padded landmark count from 64
to 16384 in steps of 64, whole gradients (T = 10, back to back, as an
optimiser runs them) are timed with each fused kernel in CTAs of both sizes
(forward 64 / 128 threads, reverse 32 / 64) and clusters of 4 to 16 CTAs
(even sizes), one kernel varied at a time; so each kernel is timed as the
gradient runs it (programmatic dependent launch, the late trigger, the state
updates).  The fastest shape of each kernel is written out, together with the
fastest cluster size for the full-size CTAs (the only ones the RK4, terminal
and planar kernels exist for).  The cluster size fixes how a target's sum is split, so the table
also fixes the rounding of every result: it is measured offline once per
GPU model and never at run time.

`--batch-shapes` times whole packed registrations for every packed launch
shape.  `--pair-loop` times the inner loops of the pair sums alone
(gs_measure_pair_loop) at 0.5 to 4 warps per scheduler, which separates the
loop's own issue limits from the fixed costs of a launch.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math

import numpy as np

from . import _lib

FWD = [(64, 2), (64, 4), (128, 2), (128, 4), (256, 1), (256, 2)]
BWD = [(64, 1), (64, 2), (128, 1), (128, 2), (256, 1)]
# fused variants: (threads per CTA, targets per thread, warp groups)
STEP_FWD = [(64, 1, 1), (64, 2, 1), (64, 4, 1), (128, 1, 1), (128, 2, 1), (128, 4, 1), (256, 1, 1), (256, 2, 1),
            (64, 1, 2), (128, 1, 2), (128, 1, 4), (256, 1, 4)]
STEP_BWD = [(32, 1, 1), (64, 1, 1), (64, 2, 1), (128, 1, 1), (128, 2, 1), (256, 1, 1), (64, 1, 2), (128, 1, 2),
            (128, 1, 4), (256, 1, 4)]
CLUSTERS = [1, 2, 4, 8, 16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[4096, 16384])
    ap.add_argument("--sigma", type=float, default=0.1)
    ap.add_argument("--reps", type=int, default=50)
    ap.add_argument("--fused-only", action="store_true", help="sweep only the fused time-step kernels")
    ap.add_argument("--policy", type=int, nargs="+", default=[-1],
                    help="cluster scheduling preferences to sweep (-1: the library's own choice)")
    ap.add_argument("--graph", action="store_true", help="time the fused kernels inside a CUDA graph")
    ap.add_argument("--clusters", type=int, nargs="+", default=CLUSTERS, help="cluster sizes of the fused sweep")
    ap.add_argument("--variants", default="all", choices=["all", "default", "small"],
                    help="default: only the (threads, R) the library picks; small: those and the one-target "
                         "variants with half the threads")
    ap.add_argument("--emit-table", metavar="PATH", help="measure the built-in step-configuration table and "
                                                           "write it to PATH")
    ap.add_argument("--instances", type=int, default=1,
                    help="--emit-table: time each shape in this many graph instantiations and keep the slowest")
    ap.add_argument("--batch-shapes", action="store_true",
                    help="time whole packed registrations (register_batch) for every packed launch shape, on the "
                         "batched distribution (N log-uniform in [500, 8000]) and on the served one "
                         "(N log-uniform in [1000, 50000])")
    ap.add_argument("--batch-count", type=int, default=128, help="--batch-shapes: problems of the batched mix")
    ap.add_argument("--batch-iters", type=int, default=20, help="--batch-shapes: L-BFGS iterations per problem")
    ap.add_argument("--pair-loop", action="store_true",
                    help="time the pair sums' inner loops alone (gs_measure_pair_loop) at 0.5 to 4 warps per "
                         "scheduler")
    args = ap.parse_args()
    import torch

    import landmark_synth as ls
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    if args.emit_table:
        emit_table(lib, dev, sms, stream, args.emit_table, args.sigma, args.instances)
        return
    if args.batch_shapes:
        batch_shapes(lib, args.batch_count, args.batch_iters)
        return
    if args.pair_loop:
        pair_loop(lib, stream)
        return
    for n in args.n:
        pr = ls.ellipsoid_pair(n, seed=0, n_bumps=8)
        rng = np.random.default_rng(1)
        q = torch.tensor(pr.q0, dtype=torch.float32, device=dev)
        p = torch.tensor(rng.normal(0, 0.01, size=(n, 3)), dtype=torch.float32, device=dev)
        a = torch.tensor(rng.normal(0, 1.0, size=(n, 3)), dtype=torch.float32, device=dev)
        b = torch.tensor(rng.normal(0, 0.01, size=(n, 3)), dtype=torch.float32, device=dev)
        P = lambda t: ctypes.c_void_p(t.data_ptr())
        npad = (n + 63) // 64 * 64
        sweeps = ((2, STEP_FWD), (3, STEP_BWD))
        if args.variants == "default":
            sweeps = ((2, [(128, 1, 1)]), (3, [(64, 1, 1)]))
        elif args.variants == "small":
            sweeps = ((2, [(64, 1, 1), (128, 1, 1)]), (3, [(32, 1, 1), (64, 1, 1)]))
        for pol in args.policy:
            _lib.check(lib.gs_set_cluster_policy(pol))
            for kind, variants in sweeps:
                for (nt, r, wg) in variants:
                    for c in args.clusters:
                        if c > nt // wg * r or c > npad // 8:
                            continue
                        ms = ctypes.c_double(0.0)
                        used = ctypes.c_int32(0)
                        st = lib.gs_time_pair_config(kind + (16 if args.graph else 0), n, args.sigma, P(q), P(p),
                                                     P(a), P(b), nt, r, wg, c, args.reps, ctypes.byref(ms),
                                                     ctypes.byref(used), stream)
                        if st != 0:
                            print(json.dumps({"n": n, "kind": kind, "threads": nt, "R": r, "groups": wg, "cluster": c,
                                              "error": lib.gs_last_error().decode()}))
                            continue
                        res = ctypes.c_int32(0)
                        lib.gs_max_active_clusters(kind - 2, nt, r, wg, c, ctypes.byref(res))
                        tiles = math.ceil(npad / (nt // wg * r))
                        print(json.dumps({"n": n, "kind": "step_fwd" if kind == 2 else "step_bwd",
                                          "threads": nt, "R": r, "groups": wg, "cluster": c, "policy": pol,
                                          "tiles": tiles,
                                          "ctas": tiles * c, "resident_ctas": res.value * c, "ms": ms.value,
                                          "gpairs_per_s": n * n / ms.value / 1e6}), flush=True)
        _lib.check(lib.gs_set_cluster_policy(-1))
        if args.fused_only:
            continue
        for kind, variants in ((0, FWD), (1, BWD)):
            for (nt, r) in variants:
                tiles = math.ceil(npad / (nt * r))
                cands = {0}
                for m in range(1, 13):
                    s = round(sms * m / tiles)
                    if 1 <= s <= npad // 8:
                        cands.add(s)
                for s in sorted(cands):
                    ms = ctypes.c_double(0.0)
                    used = ctypes.c_int32(0)
                    st = lib.gs_time_pair_config(kind, n, args.sigma, P(q), P(p), P(a), P(b), nt, r, 1, s,
                                                 args.reps, ctypes.byref(ms), ctypes.byref(used), stream)
                    if st != 0:
                        print(json.dumps({"n": n, "kind": kind, "threads": nt, "R": r, "splits": s,
                                          "error": lib.gs_last_error().decode()}))
                        continue
                    pairs = n * n
                    print(json.dumps({"n": n, "kind": "fwd" if kind == 0 else "bwd", "threads": nt, "R": r,
                                      "splits_req": s, "splits": used.value, "tiles": tiles,
                                      "ctas": tiles * used.value, "ms": ms.value,
                                      "gpairs_per_s": pairs / ms.value / 1e6}), flush=True)


# packed launch shapes (threads, cluster) per kind; a cluster must divide the CTA
BATCH_FWD = [(128, 8), (128, 4), (128, 16), (64, 8), (64, 16), (64, 4)]
BATCH_BWD = [(64, 8), (64, 4), (64, 16), (32, 8), (32, 16), (32, 4)]


# Paired FP32 instructions per source record (two landmarks) of each loop.
LOOP_INSTR = {0: 16, 1: 36}


def pair_loop(lib, stream, reps=64):
    """One JSON line per (kernel, CTA size, CTAs per SM): cycles per record per
    warp, warps per scheduler, and the FP32 pipe's share of the loop's time
    (each paired instruction holds the pipe for two cycles)."""
    for kind in (0, 1):
        for threads in (64, 128):
            for ctas in (1, 2, 3, 4, 6, 8):
                if threads * ctas > 1024:
                    continue
                cyc = ctypes.c_double(0)
                wps = threads * ctas / 128.0
                if lib.gs_measure_pair_loop(kind, threads, ctas, reps, ctypes.byref(cyc), stream) != 0:
                    print(json.dumps({"kernel": ("StepForward", "StepBackward")[kind], "threads": threads,
                                      "ctas_per_sm": ctas, "skipped": lib.gs_last_error().decode()}), flush=True)
                    continue
                print(json.dumps({"kernel": ("StepForward", "StepBackward")[kind], "threads": threads,
                                  "ctas_per_sm": ctas, "warps_per_scheduler": wps,
                                  "cycles_per_record_per_warp": round(cyc.value, 1),
                                  "fp32_pipe_share": round(2 * LOOP_INSTR[kind] * wps / cyc.value, 3)}), flush=True)


def batch_shapes(lib, count, iters, reps=3):
    """Whole packed registrations (register_batch, `iters` L-BFGS iterations
    per problem, grad_tol 0 so every shape does the same evaluations) of two
    problem mixes, for each packed launch shape: one kind varied at a time
    against the built-in shape of the other, then the best of each kind
    together.  Each line: the shape and the best of `reps` wall-clock
    times.  A packed shape is fixed per engine (gs_set_batch_config), so
    the choice never depends on the mix an engine happens to hold."""
    import time
    import torch
    import landmark_synth as ls
    from . import register_batch

    def mix_batched():
        out = []
        for r in ls.batched_requests(count, n_lo=500, n_hi=8000, sigmas=(0.05, 0.1, 0.2), first_seed=1):
            pr = ls.ellipsoid_pair(r["n"], seed=r["seed"], n_bumps=8)
            out.append(dict(q0=np.asarray(pr.q0, np.float32), target=np.asarray(pr.target, np.float32),
                            sigma=r["sigma"], lam=10.0))
        return out

    def mix_served():
        out = []
        for r in ls.poisson_trace(8, 200.0, n_lo=1000, n_hi=50000, trace_seed=0, first_seed=1001):
            pr = ls.ellipsoid_pair(r["n"], seed=r["seed"], n_bumps=8)
            out.append(dict(q0=np.asarray(pr.q0, np.float32), target=np.asarray(pr.target, np.float32),
                            sigma=0.1, lam=10.0))
        return out

    def timed(probs, fs, bs):
        _lib.check(lib.gs_set_batch_config(0, fs[0], fs[1]))
        _lib.check(lib.gs_set_batch_config(1, bs[0], bs[1]))
        best = math.inf
        for _ in range(reps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            register_batch(probs, T=20, max_iter=iters, grad_tol=0.0)
            torch.cuda.synchronize()
            best = min(best, time.perf_counter() - t0)
        return best

    try:
        for name, probs in (("batched", mix_batched()), ("served", mix_served())):
            register_batch(probs[:2], T=20, max_iter=2, grad_tol=0.0)
            base = timed(probs, BATCH_FWD[0], BATCH_BWD[0])
            res = {}
            for kind, shapes in ((0, BATCH_FWD), (1, BATCH_BWD)):
                for shp in shapes:
                    fs, bs = (shp, BATCH_BWD[0]) if kind == 0 else (BATCH_FWD[0], shp)
                    t = base if shp == (BATCH_FWD[0] if kind == 0 else BATCH_BWD[0]) else timed(probs, fs, bs)
                    res[(kind, shp)] = t
                    print(json.dumps({"mix": name, "kind": "fwd" if kind == 0 else "bwd", "threads": shp[0],
                                      "cluster": shp[1], "s": t, "vs_builtin": t / base}), flush=True)
            bf = min(BATCH_FWD, key=lambda x: res[(0, x)])
            bb = min(BATCH_BWD, key=lambda x: res[(1, x)])
            t = timed(probs, bf, bb)
            print(json.dumps({"mix": name, "best": {"fwd": bf, "bwd": bb}, "s": t, "builtin_s": base,
                              "vs_builtin": t / base}), flush=True)
    finally:
        lib.gs_set_batch_config(0, 0, 0)
        lib.gs_set_batch_config(1, 0, 0)


TABLE_SIZES = list(range(64, 16384 + 1, 64))
# (half-size CTA, full-size CTA) threads of the forward and of the reverse kernel
TABLE_FWD = (64, 128)
TABLE_BWD = (32, 64)
TABLE_CLUSTERS = (4, 6, 8, 10, 12, 14, 16)
TABLE_T = 10


def _gradient_ms(lib, prm, bufs, stream, reps, rebuild=None, instances=1):
    """Device time (ms) of one shoot_gradient call under the current step
    configuration: `reps` calls back to back between two CUDA events, as an
    optimiser issues them, after three untimed calls; the better of two such
    blocks.  With instances > 1, `rebuild()` re-applies the configuration
    (which rebuilds the cached graphs) before each further instance, and the
    slowest instance counts, so that a shape that runs in two modes is judged
    by its worse one."""
    import torch
    P = lambda t: ctypes.c_void_p(t.data_ptr())
    q, p, t, gp, gq = bufs
    run = lambda: _lib.check(lib.shoot_gradient(ctypes.byref(prm), P(q), P(p), P(t), None, P(gp), P(gq), stream))
    worst = 0.0
    for i in range(instances):
        if i:
            rebuild()
        for _ in range(3):
            run()
        best = math.inf
        for _ in range(2):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                run()
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1) / reps)
        worst = max(worst, best)
    return worst


def emit_table(lib, dev, sms, stream, path, sigma, instances=1):
    """Time every (CTA size, cluster size) of both fused kernels inside whole
    gradients at each padded size of TABLE_SIZES and write the fastest as a
    C++ table.  The forward shapes are timed with the reverse kernel at the
    size rule's shape; the reverse shapes then with the fastest forward
    shape."""
    import torch

    import landmark_synth as ls
    rows = []
    rule = {0: (128, 16), 1: (64, 8)}
    try:
        for npad in TABLE_SIZES:
            pr = ls.ellipsoid_pair(npad, seed=0, n_bumps=8)
            p0 = ls.random_momentum(npad, 0.01, seed=1)
            q, p, t = (torch.tensor(np.asarray(a, np.float32), device=dev) for a in (pr.q0, p0, pr.target))
            bufs = (q, p, t, torch.empty_like(q), torch.empty_like(q))
            prm = _lib.GsParams(N=npad, T=TABLE_T, ckpt_every=0, sigma=sigma, lambda_=10.0, lbfgs_m=10, max_iter=1,
                                grad_tol=0.0)
            reps = max(4, min(15, int(1.2e9 / npad ** 2)))
            fixed = {0: rule[0], 1: (rule[1][0], min(rule[1][1], npad // 8))}
            row = [npad]
            for kind, shapes in ((0, TABLE_FWD), (1, TABLE_BWD)):
                times = {}
                other = 1 - kind
                _lib.check(lib.gs_set_step_config(other, fixed[other][0], 1, 1, fixed[other][1]))
                for nt in shapes:
                    for c in TABLE_CLUSTERS:
                        # the rule step_config_for applies: at most one CTA of
                        # the cluster per target of the tile (M = nt with one
                        # target per thread) and at least 8 sources per CTA
                        if c > nt or c > npad // 8:
                            continue
                        apply = lambda: _lib.check(lib.gs_set_step_config(kind, nt, 1, 1, c))
                        apply()
                        times[(nt, c)] = _gradient_ms(lib, prm, bufs, stream, reps, apply, instances)
                        print(json.dumps({"npad": npad, "kind": "step_fwd" if kind == 0 else "step_bwd",
                                          "threads": nt, "cluster": c, "other": list(fixed[other]),
                                          "gradient_ms": times[(nt, c)]}), flush=True)
                best = min(times, key=times.get)
                best_full = min((k for k in times if k[0] == shapes[1]), key=times.get)
                fixed[kind] = best
                row += [best[0], best[1], best_full[1]]
            rows.append(row)
    finally:
        lib.gs_set_step_config(0, 0, 0, 0, 0)
        lib.gs_set_step_config(1, 0, 0, 0, 0)
    name = torch.cuda.get_device_name(dev)
    with open(path, "w") as f:
        f.write("// Fused step-kernel configuration per padded landmark count, measured on\n")
        f.write(f"// {name} ({sms} SMs) by\n")
        f.write("//     python -m paper_1907_04839_gb300.tune --emit-table <path>\n")
        inst = f", slowest of {instances} graph instantiations" if instances > 1 else ""
        f.write(f"// (whole gradients, T = {TABLE_T}, timed back to back{inst}).\n")
        f.write("// Columns: padded landmark count; forward CTA threads, forward cluster, cluster\n")
        f.write("// for 128-thread forward CTAs; reverse CTA threads, reverse cluster, cluster for\n")
        f.write("// 64-thread reverse CTAs.  One target per thread, one warp group.\n")
        f.write(f"constexpr int kStepTableSms = {sms};\n")
        f.write("constexpr StepRule kStepTable[] = {\n")
        for r in rows:
            f.write("    {" + ", ".join(str(v) for v in r) + "},\n")
        f.write("};\n")

if __name__ == "__main__":
    main()
