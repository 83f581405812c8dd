"""The optimiser of `register` checked from its iterates alone
(tests/lbfgs_checks.py): every accepted step is downhill, satisfies the
strong Wolfe conditions, and follows the dense BFGS inverse update of the
kept (s, y) pairs.  On the CPU the checks run on the FP64 oracle's
iterates, and they fail on iterates of a run with another memory length or
on a stretched step, which shows they can fail.  The GPU test applies them
to the library's own iterates, with (f, g) from the library's gradient, so
the GPU optimiser is pinned without reference to the oracle's line search."""
import numpy as np
import pytest

import landmark_synth as ls
import oracle
from lbfgs_checks import check_iterates

T, SIGMA, LAM, K = 10, 0.2, 10.0, 8


def case(n=128):
    pr = ls.ellipsoid_pair(n, seed=0, n_bumps=4)
    return pr.q0.astype(np.float32).astype(np.float64), pr.target.astype(np.float32).astype(np.float64)


def oracle_iterates(q0, t, m):
    xs = [np.zeros_like(q0)]
    for k in range(1, K + 1):
        r = oracle.register(q0, t, T, SIGMA, LAM, m=m, max_iter=k, grad_tol=0.0)
        assert r["iters"] == k
        xs.append(r["x"])
    return xs


def oracle_fg(q0, t):
    def fg(x):
        r = oracle.shoot_gradient(q0, x, t, T, SIGMA, LAM)
        return r["loss"], r["grad_p0"]
    return fg


def test_oracle_iterates_pass_and_the_checks_can_fail():
    q0, t = case()
    xs = oracle_iterates(q0, t, m=10)
    recs = check_iterates(xs, oracle_fg(q0, t), m=10, cos_tol=1e-9, f_slack=0.0, wolfe_slack=0.0)
    print([round(r["cos"] - 1.0, 14) for r in recs])
    # a run with memory 3 takes other directions once more than 3 pairs exist
    xs3 = oracle_iterates(q0, t, m=3)
    with pytest.raises(AssertionError, match="direction"):
        check_iterates(xs3, oracle_fg(q0, t), m=10, cos_tol=1e-9, f_slack=0.0, wolfe_slack=0.0)
    # a step stretched 4x along its own direction breaks a Wolfe condition
    bad = list(xs)
    bad[3] = xs[2] + 4.0 * (xs[3] - xs[2])
    with pytest.raises(AssertionError, match="sufficient decrease|curvature"):
        check_iterates(bad[:4], oracle_fg(q0, t), m=10, cos_tol=1e-9, f_slack=0.0, wolfe_slack=0.0)


@pytest.mark.gpu
def test_gpu_register_iterates_are_strong_wolfe_bfgs_steps():
    import paper_1907_04839_gb300 as gsh
    q0, t = case()
    q32, t32 = q0.astype(np.float32), t.astype(np.float32)
    xs = [np.zeros_like(q0)]
    for k in range(1, K + 1):
        p, info = gsh.register(q32, t32, T, SIGMA, LAM, max_iter=k, grad_tol=0.0)
        assert info["iters"] == k
        xs.append(np.asarray(p, np.float64))

    def fg(x):  # the library's own loss and gradient at the reported (FP32) momenta
        loss, gp, _ = gsh.shoot_gradient(q32, x.astype(np.float32), t32, T, SIGMA, LAM)
        return loss, np.asarray(gp, np.float64)

    # FP32 pair sums put about 1e-7 of relative noise into f and g, and the
    # reported momenta are the FP32 rounding of the FP64 iterates.
    recs = check_iterates(xs, fg, m=10, f_slack=1e-7, wolfe_slack=1e-3, cos_tol=1e-9)
    print([(r["k"], round(1.0 - r["cos"], 12)) for r in recs])


@pytest.mark.gpu
def test_gpu_packed_register_iterates_are_strong_wolfe_bfgs_steps():
    # The packed path (register_batch, and the server, which runs it) keeps a
    # line-search state machine per problem of its own; its iterates are
    # checked with (f, g) from the single-problem gradient, which differs from
    # the packed one by rounding only.
    import paper_1907_04839_gb300 as gsh
    q0, t = case()
    q32, t32 = q0.astype(np.float32), t.astype(np.float32)
    xs = [np.zeros_like(q0)]
    for k in range(1, K + 1):
        (p, info), = gsh.register_batch([dict(q0=q32, target=t32, sigma=SIGMA, lam=LAM)], T=T, max_iter=k,
                                        grad_tol=0.0)
        assert info["iters"] == k
        xs.append(np.asarray(p, np.float64))

    def fg(x):
        loss, gp, _ = gsh.shoot_gradient(q32, x.astype(np.float32), t32, T, SIGMA, LAM)
        return loss, np.asarray(gp, np.float64)

    recs = check_iterates(xs, fg, m=10, f_slack=1e-7, wolfe_slack=1e-3, cos_tol=1e-9)
    print([(r["k"], round(1.0 - r["cos"], 12)) for r in recs])
