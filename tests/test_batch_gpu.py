"""Packed batches (register_batch) and the continuous-batching server on the
GPU.  Each problem follows the same L-BFGS as register_landmarks, computed
with per-problem deterministic reductions.  A problem's result therefore
does not depend on which other problems share its launches: it is bitwise
the same alone and in a mix."""
import numpy as np
import pytest

import landmark_synth as ls
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def gs():
    import paper_1907_04839_gb300 as m
    return m


def rel(a, b):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def problems(count, seed0=1, n_lo=300, n_hi=2500):
    reqs = ls.batched_requests(count, n_lo=n_lo, n_hi=n_hi, sigmas=(0.1, 0.2), first_seed=seed0)
    out = []
    for r in reqs:
        pr = ls.ellipsoid_pair(r["n"], seed=r["seed"], n_bumps=4)
        out.append(dict(q0=pr.q0.astype(np.float32), target=pr.target.astype(np.float32), sigma=r["sigma"],
                        lam=10.0))
    return out


def test_batch_first_iterates_match_oracle():
    probs = problems(5)
    res = gs().register_batch(probs, T=8, max_iter=2, grad_tol=0.0)
    for pr, (p0, info) in zip(probs, res):
        r = oracle.register(pr["q0"].astype(np.float64), pr["target"].astype(np.float64), 8, pr["sigma"], pr["lam"],
                            max_iter=2, grad_tol=0.0)
        e = rel(p0, r["x"])
        print("N=%d sigma=%.2f p0 rel err %.2e loss %.9g / %.9g evals %d/%d" % (
            pr["q0"].shape[0], pr["sigma"], e, info["loss"], r["f"], info["evals"], r["evals"]))
        assert info["iters"] == 2 and info["evals"] == r["evals"]
        assert e < 1e-4
        assert abs(info["loss"] - r["f"]) < 1e-5 * r["f"]


def test_batch_from_a_nonzero_initial_momentum_matches_oracle():
    # The first evaluation must be at the caller's p0, not at zero.
    probs = problems(3, seed0=60, n_lo=300, n_hi=900)
    for k, pr in enumerate(probs):
        pr["p0"] = ls.random_momentum(pr["q0"].shape[0], 0.02, seed=600 + k).astype(np.float32)
    res = gs().register_batch(probs, T=8, max_iter=2, grad_tol=0.0)
    for pr, (p0, info) in zip(probs, res):
        r = oracle.register(pr["q0"].astype(np.float64), pr["target"].astype(np.float64), 8, pr["sigma"], pr["lam"],
                            p0=pr["p0"].astype(np.float64), max_iter=2, grad_tol=0.0)
        e = rel(p0, r["x"])
        print("p0 != 0: N=%d p0 rel err %.2e loss %.9g / %.9g" % (pr["q0"].shape[0], e, info["loss"], r["f"]))
        assert info["iters"] == 2 and info["evals"] == r["evals"]
        assert e < 1e-4
        assert abs(info["loss"] - r["f"]) < 1e-5 * r["f"]


def test_batch_result_is_the_same_alone_and_in_the_mix():
    probs = problems(8, seed0=20)
    mix = gs().register_batch(probs, T=6, max_iter=8, grad_tol=1e-6)
    for k in (0, 3, 7):
        alone = gs().register_batch([probs[k]], T=6, max_iter=8, grad_tol=1e-6)[0]
        assert np.array_equal(alone[0], mix[k][0])
        assert alone[1]["loss"] == mix[k][1]["loss"] and alone[1]["evals"] == mix[k][1]["evals"]


def test_server_continuous_batching_admission_and_results():
    probs = problems(6, seed0=40, n_lo=400, n_hi=1200)
    ref = gs().register_batch(probs, T=6, max_iter=6, grad_tol=1e-6)
    # A budget that holds only some requests at a time, so admission waits.
    sv = gs().Server(T=6, max_iter=6, grad_tol=1e-6, memory_budget=(64 << 20) + 2600 * 1100, max_problems=16)
    st = sv.stats()
    assert 0 < st["capacity_landmarks"] < sum(p["q0"].shape[0] for p in probs)
    ids = [sv.submit(p["q0"], p["target"], p["sigma"], p["lam"]) for p in probs[:3]]
    saw_queue = False
    for _ in range(3):
        a, q, c = sv.step()
    ids += [sv.submit(p["q0"], p["target"], p["sigma"], p["lam"]) for p in probs[3:]]
    for _ in range(500):
        a, q, c = sv.step()
        saw_queue |= q > 0
        if a == 0 and q == 0:
            break
    assert a == 0 and q == 0
    assert saw_queue
    for rid, (p0r, infr) in zip(ids, ref):
        out = sv.poll(rid)
        assert out is not None
        p0, info, lat = out
        print("server vs batch: max |dp0| %.3g loss %.12g / %.12g evals %d/%d status %d/%d" % (
            np.abs(p0 - p0r).max(), info["loss"], infr["loss"], info["evals"], infr["evals"], info["status"],
            infr["status"]))
        assert np.array_equal(p0, p0r) and info["loss"] == infr["loss"]
        assert lat[0] >= lat[1] > 0
    sv.close()


def test_server_reports_a_nonfinite_request_and_serves_the_rest():
    probs = problems(3, seed0=70, n_lo=300, n_hi=700)
    ref = gs().register_batch(probs, T=4, max_iter=3, grad_tol=1e-6)
    sv = gs().Server(T=4, max_iter=3, grad_tol=1e-6, memory_budget=256 << 20, max_problems=8)
    bad_q0 = probs[1]["q0"].copy()
    bad_q0[5, 1] = np.nan
    ids = [sv.submit(probs[0]["q0"], probs[0]["target"], probs[0]["sigma"], probs[0]["lam"]),
           sv.submit(bad_q0, probs[1]["target"], probs[1]["sigma"], probs[1]["lam"]),
           sv.submit(probs[2]["q0"], probs[2]["target"], probs[2]["sigma"], probs[2]["lam"])]
    for _ in range(200):
        a, q, c = sv.step()
        if a == 0 and q == 0:
            break
    assert a == 0 and q == 0
    with pytest.raises(gs().GShootError) as ei:
        sv.poll(ids[1])
    assert ei.value.status == -5
    for k in (0, 2):
        p0, info, _ = sv.poll(ids[k])
        assert np.array_equal(p0, ref[k][0]) and info["loss"] == ref[k][1]["loss"]
    sv.close()


def test_server_fair_schedule_finishes_small_requests_first_with_the_same_results():
    # One large request and three small ones.  Under the fair schedule the
    # small ones take more rounds per unit time and finish first; every
    # request's result is bitwise the one of the all-in-every-round schedule.
    big = problems(1, seed0=90, n_lo=3000, n_hi=3000)[0]
    small = problems(3, seed0=91, n_lo=300, n_hi=300)
    reqs = [big] + small
    finished_at = {}
    results = {}
    for sched in ("all", "fair"):
        sv = gs().Server(T=4, max_iter=12, grad_tol=0.0, memory_budget=256 << 20, max_problems=8, schedule=sched)
        ids = [sv.submit(p["q0"], p["target"], p["sigma"], p["lam"]) for p in reqs]
        rounds, fin = 0, {}
        while len(fin) < len(ids) and rounds < 2000:
            sv.step()
            rounds += 1
            for k, rid in enumerate(ids):
                if k not in fin:
                    out = sv.poll(rid)
                    if out is not None:
                        fin[k] = rounds
                        results[(sched, k)] = out
        sv.close()
        assert len(fin) == len(ids)
        finished_at[sched] = fin
        print(sched, "finished at round", fin)
    for k in range(len(reqs)):
        a, b = results[("all", k)], results[("fair", k)]
        assert np.array_equal(a[0], b[0]) and a[1]["loss"] == b[1]["loss"] and a[1]["evals"] == b[1]["evals"]
    fair, allr = finished_at["fair"], finished_at["all"]
    # all-rounds: everyone finishes within its own evaluation count of rounds
    assert all(allr[k] == results[("all", k)][1]["evals"] for k in range(len(reqs)))
    # fair: the small requests finish before the large one
    assert max(fair[k] for k in (1, 2, 3)) < fair[0]


def test_server_lanes_run_small_requests_alongside_large_ones_with_the_same_results():
    # Two large requests and four small ones under GS_SCHED_LANES (lane_split
    # 1000): the small ones run in the second engine, on their own stream and
    # host thread, during the large lane's rounds, so they finish in fewer
    # server steps than the large ones; every result is bitwise the one of a
    # packed batch (the iterates depend on neither the schedule nor the lane).
    big = problems(2, seed0=95, n_lo=6000, n_hi=8000)
    small = problems(4, seed0=96, n_lo=300, n_hi=600)
    reqs = big + small
    ref = gs().register_batch(reqs, T=4, max_iter=10, grad_tol=0.0)
    sv = gs().Server(T=4, max_iter=10, grad_tol=0.0, memory_budget=512 << 20, max_problems=8, schedule="lanes",
                     lane_split=1000)
    ids = [sv.submit(p["q0"], p["target"], p["sigma"], p["lam"]) for p in reqs]
    steps, fin, out = 0, {}, {}
    while len(fin) < len(ids) and steps < 500:
        sv.step()
        steps += 1
        for k, rid in enumerate(ids):
            if k not in fin:
                o = sv.poll(rid)
                if o is not None:
                    fin[k], out[k] = steps, o
    stats = sv.stats()
    sv.close()
    print("lanes: finished at step", fin)
    assert len(fin) == len(ids)
    for k in range(len(reqs)):
        assert np.array_equal(out[k][0], ref[k][0]) and out[k][1]["loss"] == ref[k][1]["loss"], k
        assert out[k][2][0] >= out[k][2][1] > 0
    assert max(fin[k] for k in range(2, 6)) < min(fin[0], fin[1])
    assert stats["capacity_landmarks"] > 0
