"""One template registered to a population of subjects (the shape of the
paper's Section 3.1 study) through register_batch, against the FP64 oracle's
register on each subject, and the registration reducing AverageDist and
MaxDist for every subject."""
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


def problems(n, subjects, seed, sigma=0.1, lam=10.0):
    pop = ls.population(n, subjects, seed=seed)
    q0 = pop.template.astype(np.float32)
    return [dict(q0=q0, target=t.astype(np.float32), sigma=sigma, lam=lam) for t in pop.targets]


def test_population_first_iterates_match_oracle():
    probs = problems(333, 4, seed=3)
    res = gs().register_batch(probs, T=8, max_iter=2, grad_tol=0.0)
    for pr, (p0, info) in zip(probs, res):
        r = oracle.register(pr["q0"].astype(np.float64), pr["target"].astype(np.float64), 8, pr["sigma"],
                            pr["lam"], max_iter=2, grad_tol=0.0)
        e = rel(p0, r["x"])
        print("subject: p0 rel err %.2e loss %.9g / %.9g" % (e, info["loss"], r["f"]))
        assert info["iters"] == 2 and info["evals"] == r["evals"]
        assert e < 1e-4
        assert abs(info["loss"] - r["f"]) < 1e-5 * r["f"]


def test_population_registration_reduces_distances_and_is_mix_independent():
    probs = problems(500, 5, seed=4)
    res = gs().register_batch(probs, T=10, max_iter=40, grad_tol=1e-6)
    for pr, (p0, info) in zip(probs, res):
        d0 = np.linalg.norm(pr["target"].astype(np.float64) - pr["q0"].astype(np.float64), axis=1)
        print("AverageDist %.4g -> %.4g, MaxDist %.4g -> %.4g (%d iterations)" % (
            d0.mean(), info["avg_dist"], d0.max(), info["max_dist"], info["iters"]))
        assert info["avg_dist"] < 0.5 * d0.mean()
        assert info["max_dist"] < d0.max()
    alone = gs().register_batch([probs[2]], T=10, max_iter=40, grad_tol=1e-6)[0]
    assert np.array_equal(alone[0], res[2][0]) and alone[1]["loss"] == res[2][1]["loss"]
