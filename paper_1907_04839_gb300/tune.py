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
    args = ap.parse_args()
    import torch

    import landmark_synth as ls
    lib = _lib.load()
    dev = torch.device("cuda", 0)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
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


if __name__ == "__main__":
    main()
