"""Pins for the oracle's 2-D landmarks (CPU).  The paper codes 2-D and 3-D
separately; every formula holds with 2-vectors.  A planar problem embedded
in 3-D with zero third coordinates has the same flow and gradient (every
term the third coordinate adds is an exact zero), which ties the 2-D
functions to the pinned 3-D ones; finite differences, the straight line of
one landmark and rotation equivariance pin them directly."""
import numpy as np
import pytest

import oracle

VARIANTS = [("euler", "start"), ("rk4", "start"), ("euler", "end"), ("rk4", "end")]


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def planar(n, seed, pscale=0.2, radius=0.4):
    rng = np.random.default_rng(seed)
    q = rng.uniform(-radius, radius, size=(n, 2))
    p = rng.normal(0.0, pscale, size=(n, 2))
    t = q + rng.normal(0.0, 0.05, size=(n, 2))
    return q, p, t


def embed(x):
    return np.concatenate([x, np.zeros((x.shape[0], 1))], axis=1)


def test_2d_steps_equal_the_3d_steps_of_the_embedded_problem():
    q, p, _ = planar(40, 1)
    a, b = np.random.default_rng(2).normal(size=(2, 40, 2))
    Hq, Hp = oracle.step_forward_d(q, p, 0.2)
    Hq3, Hp3 = oracle.step_forward(embed(q), embed(p), 0.2)
    assert np.array_equal(Hq, Hq3[:, :2]) and np.array_equal(Hp, Hp3[:, :2])
    assert not Hq3[:, 2].any() and not Hp3[:, 2].any()
    da, db = oracle.step_backward_d(q, p, a, b, 0.2)
    da3, db3 = oracle.step_backward(embed(q), embed(p), embed(a), embed(b), 0.2)
    assert np.array_equal(da, da3[:, :2]) and np.array_equal(db, db3[:, :2])
    # H is an OpenMP reduction, whose order of partial sums may differ by run
    h2, h3 = oracle.hamiltonian_d(q, p, 0.2), oracle.hamiltonian(embed(q), embed(p), 0.2)
    assert abs(h2 - h3) <= 1e-14 * h3


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
def test_2d_gradient_equals_the_embedded_3d_gradient(integrator, h_at):
    q, p, t = planar(60, 3)
    r2 = oracle.shoot_gradient_v(q, p, t, 5, 0.2, 10.0, integrator, h_at)
    r3 = oracle.shoot_gradient_v(embed(q), embed(p), embed(t), 5, 0.2, 10.0, integrator, h_at)
    assert abs(r2["loss"] - r3["loss"]) <= 1e-14 * r3["loss"]  # H: an OpenMP reduction
    for k in ("grad_p0", "grad_q0", "q1", "p1"):
        assert np.array_equal(r2[k], r3[k][:, :2]), k
        assert not r3[k][:, 2].any(), k


@pytest.mark.parametrize("integrator,h_at", [("euler", "start"), ("rk4", "end")])
@pytest.mark.parametrize("n,seed", [(1, 5), (4, 6), (7, 7)])
def test_2d_gradient_brute_force_finite_differences(integrator, h_at, n, seed):
    q, p, t = planar(n, seed, pscale=0.4, radius=0.25)
    T, sigma, lam, h = 4, 0.2, 10.0, 1e-5
    r = oracle.shoot_gradient_v(q, p, t, T, sigma, lam, integrator, h_at)
    L = lambda qq, pp: oracle.loss_v(qq, pp, t, T, sigma, lam, integrator, h_at)
    gp = np.zeros_like(p); gq = np.zeros_like(q)
    for i in range(n):
        for k in range(2):
            e = np.zeros_like(q); e[i, k] = h
            gp[i, k] = (L(q, p + e) - L(q, p - e)) / (2 * h)
            gq[i, k] = (L(q + e, p) - L(q - e, p)) / (2 * h)
    assert rel(r["grad_p0"], gp) < 1e-6
    assert rel(r["grad_q0"], gq) < 1e-6


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
def test_2d_single_landmark_straight_line(integrator):
    q0 = np.array([[0.3, -1.2]]); p0 = np.array([[0.7, 0.1]])
    q1, p1 = oracle.shoot_forward_v(q0, p0, 7, 0.3, integrator)
    assert np.allclose(q1, q0 + p0, rtol=0, atol=1e-14) and np.allclose(p1, p0, rtol=0, atol=1e-15)


@pytest.mark.parametrize("integrator,h_at", [("euler", "start"), ("rk4", "end")])
def test_2d_rotation_equivariance(integrator, h_at):
    q, p, t = planar(50, 8)
    c, s = np.cos(0.7), np.sin(0.7)
    R = np.array([[c, -s], [s, c]])
    t0 = np.array([0.4, -1.3])
    a = oracle.shoot_gradient_v(q, p, t, 6, 0.2, 10.0, integrator, h_at)
    b = oracle.shoot_gradient_v(q @ R.T + t0, p @ R.T, t @ R.T + t0, 6, 0.2, 10.0, integrator, h_at)
    assert abs(a["loss"] - b["loss"]) < 1e-12 * a["loss"]
    assert rel(b["grad_p0"], a["grad_p0"] @ R.T) < 1e-11
    assert rel(b["grad_q0"], a["grad_q0"] @ R.T) < 1e-11


def test_2d_register_decreases_loss():
    q, _, t = planar(30, 9)
    r = oracle.register_v(q, t, 4, 0.2, 10.0, "euler", "start", max_iter=5, grad_tol=0.0)
    tr = r["trace"][: r["iters"] + 1]
    assert r["x"].shape == (30, 2) and r["iters"] == 5 and np.all(np.diff(tr) < 0)
