"""Pins for the oracle's variants of the discretisation (CPU): the classical
fourth-order Runge-Kutta integrator with its exact discrete adjoint, and the
loss with the kinetic term at the end state (the form Algorithm 1's
pseudocode writes).  Each test ties a variant to something other than the
oracle: an exact invariant, a closed form, the convergence order, a scalar
reduction, brute-force finite differences or an independent autograd."""
import math

import numpy as np
import pytest

import landmark_synth as ls
import oracle

VARIANTS = [("rk4", "start"), ("euler", "end"), ("rk4", "end")]


def dense_K(x, y, sigma):
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    return np.exp(-d2 / (2.0 * sigma * sigma))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def small_cloud(n, seed, radius=0.3, pscale=0.3):
    rng = np.random.default_rng(seed)
    return rng.uniform(-radius, radius, size=(n, 3)), rng.normal(0.0, pscale, size=(n, 3))


@pytest.mark.parametrize("T", [1, 3, 10])
def test_rk4_single_landmark_straight_line(T):
    # N = 1: every stage has k = (p0, 0), so q(1) = q0 + p0 exactly.
    q0 = np.array([[0.3, -1.2, 2.5]]); p0 = np.array([[0.7, 0.1, -0.4]])
    q1, p1 = oracle.shoot_forward_v(q0, p0, T, 0.37, "rk4")
    assert np.allclose(p1, p0, rtol=0, atol=1e-15)
    assert np.allclose(q1, q0 + p0, rtol=0, atol=1e-13)


def test_rk4_total_momentum_conserved():
    pr = ls.ellipsoid_pair(200, seed=2, n_bumps=4)
    p0 = ls.random_momentum(200, 0.05, seed=3)
    for T in (1, 4, 9):
        _, p1 = oracle.shoot_forward_v(pr.q0, p0, T, 0.2, "rk4")
        assert np.abs(p1.sum(0) - p0.sum(0)).max() < 1e-13 * np.abs(p0).sum()


def test_rk4_energy_and_angular_momentum_drift_fourth_order():
    # H and sum q x p are exact invariants of Eq. 2.  The RK4 drift of the
    # angular momentum falls by 2^4 = 16 when dt halves; the energy drift
    # falls at least as fast and approaches the same rate.
    rng = np.random.default_rng(4)
    q0, p0 = rng.uniform(-0.4, 0.4, size=(24, 3)), rng.normal(0.0, 0.2, size=(24, 3))
    sigma = 0.3
    H0 = oracle.hamiltonian(q0, p0, sigma)
    J0 = np.cross(q0, p0).sum(0)
    dH, dJ = [], []
    for T in (10, 20, 40, 80, 160):
        q1, p1 = oracle.shoot_forward_v(q0, p0, T, sigma, "rk4")
        dH.append(abs(oracle.hamiltonian(q1, p1, sigma) - H0))
        dJ.append(np.linalg.norm(np.cross(q1, p1).sum(0) - J0))
    oJ = [math.log2(a / b) for a, b in zip(dJ[:-1], dJ[1:])]
    oH = [math.log2(a / b) for a, b in zip(dH[:-1], dH[1:])]
    print("orders: angular momentum", oJ, "energy", oH)
    assert all(abs(o - 4.0) < 0.1 for o in oJ[1:]) and abs(oJ[-1] - 4.0) < 0.05
    assert all(o > 3.95 for o in oH) and oH[-1] < 4.4 and all(a > b for a, b in zip(oH[:-1], oH[1:]))


def test_rk4_two_body_head_on_scalar_recursion():
    # p1 = -p2 = P e_x, q1 = -q2 = (r/2) e_x stay on the x axis at every stage:
    # RK4 on (r, P) with dr/dt = 2P(1 - g(r)), dP/dt = -s P^2 g(r) r.
    sigma, T, r, P = 0.4, 7, 0.5, 0.8
    s = 1.0 / sigma ** 2
    q0 = np.array([[r / 2, 0, 0], [-r / 2, 0, 0]]); p0 = np.array([[P, 0, 0], [-P, 0, 0]])
    q1, p1 = oracle.shoot_forward_v(q0, p0, T, sigma, "rk4")

    def f(r, P):
        g = math.exp(-r * r / (2 * sigma * sigma))
        return 2 * P * (1 - g), -s * P * P * g * r

    dt = 1.0 / T
    for _ in range(T):
        a1, b1 = f(r, P)
        a2, b2 = f(r + dt / 2 * a1, P + dt / 2 * b1)
        a3, b3 = f(r + dt / 2 * a2, P + dt / 2 * b2)
        a4, b4 = f(r + dt * a3, P + dt * b3)
        r, P = r + dt / 6 * (a1 + 2 * a2 + 2 * a3 + a4), P + dt / 6 * (b1 + 2 * b2 + 2 * b3 + b4)
    assert abs((q1[0, 0] - q1[1, 0]) - r) < 1e-14
    assert abs(p1[0, 0] - P) < 1e-14 and abs(p1[1, 0] + P) < 1e-14


def test_euler_start_variant_is_the_plain_method():
    pr = ls.ellipsoid_pair(64, seed=8, n_bumps=4)
    p0 = ls.random_momentum(64, 0.05, seed=9)
    a = oracle.shoot_gradient(pr.q0, p0, pr.target, 5, 0.2, 10.0)
    b = oracle.shoot_gradient_v(pr.q0, p0, pr.target, 5, 0.2, 10.0, "euler", "start")
    assert a["loss"] == b["loss"]
    assert np.array_equal(a["grad_p0"], b["grad_p0"]) and np.array_equal(a["grad_q0"], b["grad_q0"])


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
def test_variant_gradient_closed_form_at_zero_momentum(integrator, h_at):
    # p0 = 0: the flow is static for either integrator, H = 0 at both ends,
    # and the adjoint gives dL/dp0 = 2 lambda K(q0)(q0 - t), dL/dq0 = 2 lambda (q0 - t).
    pr = ls.ellipsoid_pair(200, seed=1, n_bumps=4)
    lam, sigma = 10.0, 0.2
    for T in (1, 6):
        r = oracle.shoot_gradient_v(pr.q0, np.zeros_like(pr.q0), pr.target, T, sigma, lam, integrator, h_at)
        resid = pr.q0 - pr.target
        assert abs(r["loss"] - lam * np.sum(resid ** 2)) < 1e-12 * r["loss"]
        assert rel(r["grad_p0"], 2 * lam * dense_K(pr.q0, pr.q0, sigma) @ resid) < 1e-12
        assert rel(r["grad_q0"], 2 * lam * resid) < 1e-12


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
@pytest.mark.parametrize("n,seed", [(1, 40), (3, 41), (8, 42)])
def test_variant_gradient_brute_force_finite_differences(integrator, h_at, n, seed):
    q, p = small_cloud(n, seed, radius=0.25, pscale=0.4)
    t = q + np.random.default_rng(seed + 100).normal(0, 0.1, size=q.shape)
    T, sigma, lam, h = 4, 0.2, 10.0, 1e-5
    r = oracle.shoot_gradient_v(q, p, t, T, sigma, lam, integrator, h_at)
    L = lambda qq, pp: oracle.loss_v(qq, pp, t, T, sigma, lam, integrator, h_at)
    assert abs(r["loss"] - L(q, p)) < 1e-13 * abs(r["loss"])
    gp = np.zeros_like(p); gq = np.zeros_like(q)
    for i in range(n):
        for k in range(3):
            e = np.zeros_like(q); e[i, k] = h
            gp[i, k] = (L(q, p + e) - L(q, p - e)) / (2 * h)
            gq[i, k] = (L(q + e, p) - L(q - e, p)) / (2 * h)
    assert rel(r["grad_p0"], gp) < 1e-6
    assert rel(r["grad_q0"], gq) < 1e-6


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
def test_variant_gradient_matches_independent_autograd(integrator, h_at):
    # torch autograd (FP64, CPU) of a loop written from Eq. 1 and the
    # integrator's definition: independent of the hand-derived adjoint.
    torch = pytest.importorskip("torch")
    pr = ls.ellipsoid_pair(96, seed=13, n_bumps=4)
    p0n = ls.random_momentum(96, 0.1, seed=14)
    T, sigma, lam = 5, 0.25, 10.0

    def H(q, p):
        d2 = ((q[:, None, :] - q[None, :, :]) ** 2).sum(-1)
        return 0.5 * (p * (torch.exp(-d2 / (2 * sigma * sigma)) @ p)).sum()

    def f(q, p):
        gq, gp = torch.autograd.grad(H(q, p), (q, p), create_graph=True)
        return gp, -gq

    q0 = torch.tensor(pr.q0, dtype=torch.float64, requires_grad=True)
    p0 = torch.tensor(p0n, dtype=torch.float64, requires_grad=True)
    tgt = torch.tensor(pr.target, dtype=torch.float64)
    q, p, dt = q0, p0, 1.0 / T
    for _ in range(T):
        if integrator == "euler":
            a, b = f(q, p)
            q, p = q + dt * a, p + dt * b
        else:
            a1, b1 = f(q, p)
            a2, b2 = f(q + dt / 2 * a1, p + dt / 2 * b1)
            a3, b3 = f(q + dt / 2 * a2, p + dt / 2 * b2)
            a4, b4 = f(q + dt * a3, p + dt * b3)
            q, p = q + dt / 6 * (a1 + 2 * a2 + 2 * a3 + a4), p + dt / 6 * (b1 + 2 * b2 + 2 * b3 + b4)
    L = (H(q, p) if h_at == "end" else H(q0, p0)) + lam * ((q - tgt) ** 2).sum()
    L.backward()
    r = oracle.shoot_gradient_v(pr.q0, p0n, pr.target, T, sigma, lam, integrator, h_at)
    assert abs(r["loss"] - L.item()) < 1e-12 * abs(L.item())
    assert rel(r["grad_p0"], p0.grad.numpy()) < 1e-10
    assert rel(r["grad_q0"], q0.grad.numpy()) < 1e-10


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
def test_variant_rigid_motion_invariance(integrator, h_at):
    pr = ls.ellipsoid_pair(100, seed=15, n_bumps=4)
    p0 = ls.random_momentum(100, 0.05, seed=16)
    A = np.random.default_rng(17).normal(size=(3, 3))
    R, Rr = np.linalg.qr(A)
    R = R * np.sign(np.diag(Rr))
    if np.linalg.det(R) < 0:
        R[:, 0] = -R[:, 0]
    t0 = np.array([0.3, -2.0, 1.1])
    a = oracle.shoot_gradient_v(pr.q0, p0, pr.target, 6, 0.2, 10.0, integrator, h_at)
    b = oracle.shoot_gradient_v(pr.q0 @ R.T + t0, p0 @ R.T, pr.target @ R.T + t0, 6, 0.2, 10.0, integrator, h_at)
    assert abs(a["loss"] - b["loss"]) < 1e-12 * a["loss"]
    assert rel(b["grad_p0"], a["grad_p0"] @ R.T) < 1e-11
    assert rel(b["grad_q0"], a["grad_q0"] @ R.T) < 1e-11


def test_kinetic_term_at_end_is_H_of_the_end_state():
    # lambda = 0: the loss is H(p(1), q(1)); RK4 keeps it within its
    # fourth-order drift of H(p0, q0).
    q, p = small_cloud(20, 18, radius=0.4, pscale=0.15)
    r = oracle.shoot_gradient_v(q, p, np.zeros_like(q), 16, 0.3, 0.0, "rk4", "end")
    d2 = ((r["q1"][:, None, :] - r["q1"][None, :, :]) ** 2).sum(-1)
    H1 = 0.5 * float(np.sum(r["p1"] * (np.exp(-d2 / (2 * 0.3 ** 2)) @ r["p1"])))
    assert abs(r["loss"] - H1) < 1e-13 * H1
    d2 = ((q[:, None, :] - q[None, :, :]) ** 2).sum(-1)
    H0 = 0.5 * float(np.sum(p * (np.exp(-d2 / (2 * 0.3 ** 2)) @ p)))
    assert abs(H1 - H0) < 1e-5 * H0


def test_register_variant_decreases_loss():
    pr = ls.ellipsoid_pair(64, seed=19, n_bumps=4)
    r = oracle.register_v(pr.q0, pr.target, 4, 0.2, 10.0, "rk4", "end", max_iter=5, grad_tol=0.0)
    tr = r["trace"][: r["iters"] + 1]
    assert r["iters"] == 5 and np.all(np.diff(tr) < 0)
