"""The oracle's L-BFGS (the optimiser `register` runs, Section 2.1 and
Algorithm 1's outer loop) observed from outside through every evaluation it
makes, on objectives written here.  Two properties fix it independently of
its code:

* every accepted step satisfies the strong Wolfe conditions with c1 = 1e-4,
  c2 = 0.9 along a descent direction (the definition of the line search it
  claims to run);
* every search direction is -H_k g_k, with H_k the inverse-Hessian
  approximation built by applying the BFGS inverse update, as a dense matrix,
  to gamma_k I for each of the last m stored pairs (s, y), oldest first:
  the matrix the two-loop recursion applies without forming it.  The first
  trial step is 1/||g_0|| at the first iteration and 1 afterwards.

The GPU `register` matches the oracle's iterates (tests/test_register_gpu.py),
so these pins carry over to it."""
import numpy as np
import pytest

import oracle

C1, C2 = 1e-4, 0.9


def rosenbrock(x):
    a, b = x[::2], x[1::2]
    f = float(np.sum(100.0 * (b - a * a) ** 2 + (1.0 - a) ** 2))
    g = np.zeros_like(x)
    g[::2] = -400.0 * a * (b - a * a) - 2.0 * (1.0 - a)
    g[1::2] = 200.0 * (b - a * a)
    return f, g


def convex(n, seed):
    # 1/2 x^T A x - b^T x + sum_i log(1 + exp(c_i . x)): smooth, strictly convex
    rng = np.random.default_rng(seed)
    M = rng.normal(size=(n, n))
    A = M @ M.T / n + 0.1 * np.eye(n)
    b = rng.normal(size=n)
    Cm = rng.normal(size=(3 * n, n)) / np.sqrt(n)

    def fg(x):
        z = Cm @ x
        f = 0.5 * x @ A @ x - b @ x + float(np.sum(np.logaddexp(0.0, z)))
        g = A @ x - b + Cm.T @ (1.0 / (1.0 + np.exp(-z)))
        return f, g
    return fg


def run(fg, x0, m, max_iter):
    evals = []

    def rec(x):
        f, g = fg(x)
        evals.append((x.copy(), f, np.asarray(g, dtype=np.float64).copy()))
        return f, g

    res = oracle.lbfgs_callback(rec, x0, m=m, max_iter=max_iter, grad_tol=1e-8)
    return res, evals


def iterations(evals, g0norm):
    """Split the evaluation sequence into line searches: each starts at the
    current iterate x_k with a first trial x_k + a1 d_k (a1 = 1/||g0|| at the
    first iteration, 1 afterwards), continues along that ray, and ends at the
    accepted trial, which the next iteration starts from."""
    out = []
    base, k, i = 0, 0, 1
    while i < len(evals):
        xk = evals[base][0]
        a1 = 1.0 / g0norm if k == 0 else 1.0
        d = (evals[i][0] - xk) / a1
        dd = float(d @ d)
        steps = [(i, a1)]
        j = i + 1
        while j < len(evals):
            v = evals[j][0] - xk
            a = float(v @ d) / dd
            if np.linalg.norm(v - a * d) > 1e-9 * max(1.0, np.linalg.norm(v)):
                break
            steps.append((j, a))
            j += 1
        acc, a_acc = steps[-1]
        out.append(dict(base=base, d=d, acc=acc, a=a_acc, trials=len(steps)))
        base, k, i = acc, k + 1, j
    return out


def dense_lbfgs_direction(g, pairs, m):
    """-H g with H the BFGS inverse update of gamma I over the last m pairs."""
    n = g.size
    use = pairs[-m:]
    if not use:
        return -g
    s_l, y_l = use[-1]
    H = (s_l @ y_l) / (y_l @ y_l) * np.eye(n)
    for s, y in use:
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return -H @ g


@pytest.mark.parametrize("case", ["rosenbrock4", "rosenbrock8", "convex20"])
def test_lbfgs_steps_are_strong_wolfe_and_directions_are_bfgs(case):
    m = 5
    if case.startswith("rosenbrock"):
        n = int(case[len("rosenbrock"):])
        fg, x0 = rosenbrock, np.tile([-1.2, 1.0], n // 2)
    else:
        fg, x0 = convex(20, 3), np.zeros(20)
    res, evals = run(fg, x0, m, 200)
    assert res["status"] == 0 and res["evals"] == len(evals)
    its = iterations(evals, np.linalg.norm(evals[0][2]))
    assert len(its) == res["iters"]
    assert any(it["trials"] > 1 for it in its) or case == "convex20"  # the search does more than accept
    pairs = []
    for k, it in enumerate(its):
        xb, fb, gb = evals[it["base"]]
        xa, fa, ga = evals[it["acc"]]
        d, a = it["d"], it["a"]
        slope0 = float(gb @ d)
        assert slope0 < 0.0, (case, k)
        assert fa <= fb + C1 * a * slope0 + 1e-12 * abs(fb), (case, k, "sufficient decrease")
        assert abs(float(ga @ d)) <= C2 * abs(slope0) * (1 + 1e-12), (case, k, "curvature")
        ref = dense_lbfgs_direction(gb, pairs, m)
        assert np.linalg.norm(d - ref) <= 1e-7 * np.linalg.norm(ref), (case, k, "direction")
        s, y = xa - xb, ga - gb
        if s @ y > 1e-12 * np.sqrt((s @ s) * (y @ y)):
            pairs.append((s, y))
    assert np.linalg.norm(evals[its[-1]["acc"]][2]) <= 1e-8 * np.linalg.norm(evals[0][2])
