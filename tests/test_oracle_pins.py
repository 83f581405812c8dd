"""Pins for the FP64 oracle: each test ties one oracle function to something
other than the oracle itself -- a closed form, an exact invariant of Eq. 2, a
textbook definition evaluated with numpy/BLAS, brute-force finite differences,
or an independent autograd of the Euler loop.  CPU only."""
import math

import numpy as np
import pytest

import landmark_synth as ls
import oracle


def dense_K(x, y, sigma):
    """Gaussian kernel matrix of Section 2.1 between point sets x (M,3), y (N,3)."""
    d2 = ((x[:, None, :] - y[None, :, :]) ** 2).sum(-1)
    return np.exp(-d2 / (2.0 * sigma * sigma))


def H_dense(q, p, sigma):
    """Eq. 1 as a dense quadratic form 1/2 p^T K(q) p (BLAS)."""
    K = dense_K(q, q, sigma)
    return 0.5 * float(np.sum(p * (K @ p)))


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


def small_cloud(n, seed, radius=0.3, pscale=0.3):
    rng = np.random.default_rng(seed)
    q = rng.uniform(-radius, radius, size=(n, 3))
    p = rng.normal(0.0, pscale, size=(n, 3))
    return q, p


# ---------------------------------------------------------------- forward

@pytest.mark.parametrize("T", [1, 3, 10, 40])
def test_single_landmark_straight_line(T):
    # N = 1: g = 1 and d = 0, so p is constant and q(1) = q0 + p0 (T dt = 1).
    q0 = np.array([[0.3, -1.2, 2.5]])
    p0 = np.array([[0.7, 0.1, -0.4]])
    q1, p1, tq, tp = oracle.shoot_forward(q0, p0, T, 0.37, trajectory=True)
    assert np.allclose(p1, p0, rtol=0, atol=1e-15)
    assert np.allclose(q1, q0 + p0, rtol=0, atol=1e-13)
    for k in range(T + 1):  # q(t) = q0 + p0 t at every step
        assert np.allclose(tq[k], q0 + p0 * (k / T), rtol=0, atol=1e-13)


def test_hp_is_dense_K_matvec():
    q, p = small_cloud(300, 1)
    Hq, Hp = oracle.step_forward(q, p, 0.2)
    assert rel(Hp, dense_K(q, q, 0.2) @ p) < 1e-13


def test_hq_hp_are_partial_derivatives_of_H():
    # Eq. 2: Hp = dH/dp and Hq = dH/dq, checked by central differences of the
    # dense quadratic form of Eq. 1.
    q, p = small_cloud(7, 2)
    sigma, h = 0.25, 1e-5
    Hq, Hp = oracle.step_forward(q, p, sigma)
    fq = np.zeros_like(q); fp = np.zeros_like(p)
    for i in range(q.shape[0]):
        for k in range(3):
            e = np.zeros_like(q); e[i, k] = h
            fq[i, k] = (H_dense(q + e, p, sigma) - H_dense(q - e, p, sigma)) / (2 * h)
            fp[i, k] = (H_dense(q, p + e, sigma) - H_dense(q, p - e, sigma)) / (2 * h)
    assert rel(Hp, fp) < 1e-8
    assert rel(Hq, fq) < 1e-8


def test_row_restricted_steps_match_dense_products():
    # The row-restricted entry points compute the same sums for the chosen
    # targets: Hp rows against the dense K matvec (BLAS), and every row
    # against the full-set sweep.
    q, p = small_cloud(500, 30)
    rng = np.random.default_rng(31)
    a = rng.normal(size=q.shape); b = rng.normal(size=q.shape)
    rows = np.array([0, 7, 499, 250, 7])
    Hq, Hp = oracle.step_forward_rows(q, p, 0.2, rows)
    assert rel(Hp, (dense_K(q, q, 0.2) @ p)[rows]) < 1e-13
    Hq_all, Hp_all = oracle.step_forward(q, p, 0.2)
    assert np.array_equal(Hq, Hq_all[rows]) and np.array_equal(Hp, Hp_all[rows])
    da, db = oracle.step_backward_rows(q, p, a, b, 0.2, rows)
    da_all, db_all = oracle.step_backward(q, p, a, b, 0.2)
    assert np.array_equal(da, da_all[rows]) and np.array_equal(db, db_all[rows])


def test_hamiltonian_matches_dense_quadratic_form():
    q, p = small_cloud(200, 3)
    assert abs(oracle.hamiltonian(q, p, 0.15) - H_dense(q, p, 0.15)) < 1e-12 * abs(H_dense(q, p, 0.15))


def test_total_momentum_conserved():
    # sum_i Hq_i = 0 by antisymmetry of d_ij, so sum_i p_i is constant.
    pr = ls.ellipsoid_pair(256, seed=0, n_bumps=4)
    p0 = ls.random_momentum(256, 0.05, seed=5)
    q1, p1, tq, tp = oracle.shoot_forward(pr.q0, p0, 10, 0.2, trajectory=True)
    scale = np.abs(tp).sum(axis=1).max()
    for k in range(11):
        assert np.abs(tp[k].sum(0) - p0.sum(0)).max() < 1e-13 * scale
    Hq, _ = oracle.step_forward(pr.q0, p0, 0.2)
    assert np.abs(Hq.sum(0)).max() < 1e-13 * np.abs(Hq).sum()


def test_energy_and_angular_momentum_drift_first_order():
    # H and sum q x p are exact invariants of Eq. 2; explicit Euler drifts at
    # first order, so the drift halves when dt halves.
    q0, p0 = small_cloud(24, 4, radius=0.4, pscale=0.2)
    sigma = 0.3
    H0 = oracle.hamiltonian(q0, p0, sigma)
    J0 = np.cross(q0, p0).sum(0)
    dH, dJ = [], []
    for T in (20, 40, 80, 160, 320):
        q1, p1 = oracle.shoot_forward(q0, p0, T, sigma)
        dH.append(abs(oracle.hamiltonian(q1, p1, sigma) - H0))
        dJ.append(np.linalg.norm(np.cross(q1, p1).sum(0) - J0))
    for d in (dH, dJ):
        ratios = [a / b for a, b in zip(d[:-1], d[1:])]
        assert all(1.9 < x < 2.15 for x in ratios)
        assert abs(ratios[-1] - 2.0) < 0.03  # tends to 2: first order


def test_two_body_head_on_scalar_recursion():
    # p1 = -p2 = P e_x, q1 = -q2 = (r/2) e_x stay on the x axis:
    # dr/dt = 2P(1 - g(r)), dP/dt = -s P^2 g(r) r.
    sigma, T, r, P = 0.4, 25, 0.5, 0.8
    s = 1.0 / sigma ** 2
    q0 = np.array([[r / 2, 0, 0], [-r / 2, 0, 0]])
    p0 = np.array([[P, 0, 0], [-P, 0, 0]])
    q1, p1 = oracle.shoot_forward(q0, p0, T, sigma)
    dt = 1.0 / T
    for _ in range(T):
        g = math.exp(-r * r / (2 * sigma * sigma))
        r, P = r + dt * 2 * P * (1 - g), P - dt * s * P * P * g * r
    assert abs((q1[0, 0] - q1[1, 0]) - r) < 1e-14
    assert abs(p1[0, 0] - P) < 1e-14 and abs(p1[1, 0] + P) < 1e-14
    assert np.abs(q1[:, 1:]).max() == 0.0 and np.abs(p1[:, 1:]).max() == 0.0


def test_velocity_field_eq4():
    q, p = small_cloud(100, 6)
    x = np.random.default_rng(7).uniform(-0.5, 0.5, size=(57, 3))
    v = oracle.velocity(x, q, p, 0.2)
    assert rel(v, dense_K(x, q, 0.2) @ p) < 1e-13
    # at the landmarks themselves the field equals dq/dt = Hp
    _, Hp = oracle.step_forward(q, p, 0.2)
    assert rel(oracle.velocity(q, q, p, 0.2), Hp) < 1e-13


def test_flow_points_carries_landmarks_exactly_with_q():
    # A landmark used as a point moves with v(q_i) = Hp_i, i.e. exactly as the
    # landmark does through the T Euler steps.
    q, p = small_cloud(60, 21)
    T, sigma = 7, 0.2
    q1, _ = oracle.shoot_forward(q, p, T, sigma)
    x1 = oracle.flow_points(q, p, q, T, sigma)
    assert np.max(np.abs(x1 - q1)) <= 1e-14 * np.max(np.abs(q1))


def test_flow_points_far_points_do_not_move():
    # g underflows to exactly 0 beyond ~39 sigma, so the velocity is 0.
    q, p = small_cloud(30, 22)
    x0 = np.array([[60.0, 0.0, 0.0], [0.0, -45.0, 3.0]])
    x1 = oracle.flow_points(q, p, x0, 5, 0.2)
    assert np.array_equal(x1, x0)


def test_flow_points_single_landmark_scalar_recursion():
    # One landmark: q(t) = q0 + p0 t exactly.  A point offset by delta,
    # perpendicular to p0, keeps that perpendicular offset and its separation
    # s along p0 follows s_{k+1} = s_k + dt (g(r_k) - 1) |p0|, r_k^2 = |delta|^2 + s_k^2.
    q0 = np.array([[0.2, -0.1, 0.4]])
    p0 = np.array([[0.6, 0.0, 0.0]])
    delta = np.array([0.0, 0.15, -0.05])
    T, sigma = 25, 0.3
    x1 = oracle.flow_points(q0, p0, q0 + delta[None, :], T, sigma)
    dt, s = 1.0 / T, 0.0
    d2 = float(delta @ delta)
    for _ in range(T):
        s += dt * (math.exp(-(d2 + s * s) / (2 * sigma * sigma)) - 1.0) * 0.6
    expect = q0[0] + p0[0] + delta + np.array([s, 0.0, 0.0])
    assert np.max(np.abs(x1[0] - expect)) < 1e-14


def test_flow_points_rigid_motion_equivariance():
    q, p = small_cloud(40, 23)
    x0 = np.random.default_rng(24).uniform(-0.4, 0.4, size=(25, 3))
    A = np.random.default_rng(25).normal(size=(3, 3))
    Rm, _ = np.linalg.qr(A)
    t0 = np.array([0.3, -0.7, 1.1])
    x1 = oracle.flow_points(q, p, x0, 6, 0.25)
    y1 = oracle.flow_points(q @ Rm.T + t0, p @ Rm.T, x0 @ Rm.T + t0, 6, 0.25)
    assert rel(y1, x1 @ Rm.T + t0) < 1e-12


# ---------------------------------------------------------------- backward

def test_step_backward_is_transposed_jacobian():
    # <(alpha, beta), J v> = <StepBackward(alpha, beta), v> for the map
    # f(q, p) = (Hp, -Hq), with J v by central differences of StepForward.
    rng = np.random.default_rng(8)
    q, p = small_cloud(40, 9)
    a = rng.normal(size=q.shape); b = rng.normal(size=q.shape)
    vq = rng.normal(size=q.shape); vp = rng.normal(size=q.shape)
    sigma, h = 0.25, 1e-6
    Hq1, Hp1 = oracle.step_forward(q + h * vq, p + h * vp, sigma)
    Hq2, Hp2 = oracle.step_forward(q - h * vq, p - h * vp, sigma)
    Jv_q = (Hp1 - Hp2) / (2 * h)
    Jv_p = -(Hq1 - Hq2) / (2 * h)
    lhs = np.sum(a * Jv_q) + np.sum(b * Jv_p)
    da, db = oracle.step_backward(q, p, a, b, sigma)
    rhs = np.sum(da * vq) + np.sum(db * vp)
    assert abs(lhs - rhs) < 1e-7 * (abs(lhs) + 1)


def test_adjoint_alpha_sum_conserved():
    # sum_i dalpha_i = 0 by antisymmetry, so sum_i alpha_i is constant.
    rng = np.random.default_rng(10)
    q, p = small_cloud(64, 11)
    a = rng.normal(size=q.shape); b = rng.normal(size=q.shape)
    da, db = oracle.step_backward(q, p, a, b, 0.2)
    assert np.abs(da.sum(0)).max() < 1e-12 * np.abs(da).sum()


def test_gradient_closed_form_at_zero_momentum():
    # p0 = 0: the flow is static, L = lambda ||q0 - t||^2,
    # dL/dp0 = 2 lambda K(q0) (q0 - t), dL/dq0 = 2 lambda (q0 - t), any T.
    pr = ls.ellipsoid_pair(256, seed=0, n_bumps=4)
    lam, sigma = 10.0, 0.2
    for T in (1, 10):
        r = oracle.shoot_gradient(pr.q0, np.zeros_like(pr.q0), pr.target, T, sigma, lam)
        resid = pr.q0 - pr.target
        assert abs(r["loss"] - lam * np.sum(resid ** 2)) < 1e-12 * r["loss"]
        assert rel(r["grad_p0"], 2 * lam * dense_K(pr.q0, pr.q0, sigma) @ resid) < 1e-12
        assert rel(r["grad_q0"], 2 * lam * resid) < 1e-12


def test_gradient_lambda_zero_is_dH():
    # lambda = 0: L = H(p0, q0), so dL/dp0 = K p0 and dL/dq0 = dH/dq0.
    q, p = small_cloud(6, 12)
    sigma, h = 0.25, 1e-5
    r = oracle.shoot_gradient(q, p, np.zeros_like(q), 7, sigma, 0.0)
    assert abs(r["loss"] - H_dense(q, p, sigma)) < 1e-13
    assert rel(r["grad_p0"], dense_K(q, q, sigma) @ p) < 1e-13
    fq = np.zeros_like(q)
    for i in range(q.shape[0]):
        for k in range(3):
            e = np.zeros_like(q); e[i, k] = h
            fq[i, k] = (H_dense(q + e, p, sigma) - H_dense(q - e, p, sigma)) / (2 * h)
    assert rel(r["grad_q0"], fq) < 1e-8


def test_gradient_translation_identity():
    # Translating q0 and target together leaves L unchanged, which forces
    # sum_i dL/dq0_i = 2 lambda sum_i (q1_i - t_i).
    pr = ls.ellipsoid_pair(128, seed=3, n_bumps=4)
    p0 = ls.random_momentum(128, 0.05, seed=4)
    r = oracle.shoot_gradient(pr.q0, p0, pr.target, 8, 0.2, 10.0)
    lhs = r["grad_q0"].sum(0)
    rhs = 2 * 10.0 * (r["q1"] - pr.target).sum(0)
    assert np.abs(lhs - rhs).max() < 1e-10 * np.abs(r["grad_q0"]).sum()


def _rotation(seed):
    A = np.random.default_rng(seed).normal(size=(3, 3))
    Q, R = np.linalg.qr(A)
    Q = Q * np.sign(np.diag(R))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    return Q


def test_rigid_motion_invariance():
    pr = ls.ellipsoid_pair(128, seed=5, n_bumps=4)
    p0 = ls.random_momentum(128, 0.05, seed=6)
    R, t0 = _rotation(13), np.array([0.3, -2.0, 1.1])
    a = oracle.shoot_gradient(pr.q0, p0, pr.target, 8, 0.2, 10.0)
    b = oracle.shoot_gradient(pr.q0 @ R.T + t0, p0 @ R.T, pr.target @ R.T + t0, 8, 0.2, 10.0)
    assert abs(a["loss"] - b["loss"]) < 1e-12 * a["loss"]
    assert rel(b["grad_p0"], a["grad_p0"] @ R.T) < 1e-11
    assert rel(b["grad_q0"], a["grad_q0"] @ R.T) < 1e-11
    assert rel(b["q1"], a["q1"] @ R.T + t0) < 1e-12


@pytest.mark.parametrize("n,seed", [(1, 20), (2, 21), (5, 22), (8, 23)])
def test_gradient_brute_force_finite_differences(n, seed):
    q, p = small_cloud(n, seed, radius=0.25, pscale=0.4)
    t = q + np.random.default_rng(seed + 100).normal(0, 0.1, size=q.shape)
    T, sigma, lam, h = 6, 0.2, 10.0, 1e-5
    r = oracle.shoot_gradient(q, p, t, T, sigma, lam)
    gp = np.zeros_like(p); gq = np.zeros_like(q)
    for i in range(n):
        for k in range(3):
            e = np.zeros_like(q); e[i, k] = h
            gp[i, k] = (oracle.loss(q, p + e, t, T, sigma, lam) - oracle.loss(q, p - e, t, T, sigma, lam)) / (2 * h)
            gq[i, k] = (oracle.loss(q + e, p, t, T, sigma, lam) - oracle.loss(q - e, p, t, T, sigma, lam)) / (2 * h)
    assert rel(r["grad_p0"], gp) < 1e-6
    assert rel(r["grad_q0"], gq) < 1e-6


def test_gradient_directional_fd_medium():
    # Directional central differences on a mid-size ellipsoid problem.
    pr = ls.ellipsoid_pair(512, seed=7, n_bumps=8)
    p0 = ls.random_momentum(512, 0.02, seed=8)
    T, sigma, lam, h = 5, 0.1, 10.0, 1e-5
    r = oracle.shoot_gradient(pr.q0, p0, pr.target, T, sigma, lam)
    rng = np.random.default_rng(9)
    for _ in range(3):
        v = rng.normal(size=p0.shape); v /= np.linalg.norm(v)
        fd = (oracle.loss(pr.q0, p0 + h * v, pr.target, T, sigma, lam)
              - oracle.loss(pr.q0, p0 - h * v, pr.target, T, sigma, lam)) / (2 * h)
        an = float(np.sum(r["grad_p0"] * v))
        assert abs(fd - an) <= 1e-6 * np.linalg.norm(r["grad_p0"])


def test_gradient_matches_independent_autograd():
    # torch autograd (FP64, CPU) of an Euler loop whose Hq, Hp come from
    # differentiating Eq. 1 itself: independent of the hand-derived adjoint.
    torch = pytest.importorskip("torch")
    pr = ls.ellipsoid_pair(96, seed=11, n_bumps=4)
    p0n = ls.random_momentum(96, 0.1, seed=12)
    T, sigma, lam = 6, 0.25, 10.0

    def H(q, p):
        d2 = ((q[:, None, :] - q[None, :, :]) ** 2).sum(-1)
        return 0.5 * (p * (torch.exp(-d2 / (2 * sigma * sigma)) @ p)).sum()

    q0 = torch.tensor(pr.q0, dtype=torch.float64, requires_grad=True)
    p0 = torch.tensor(p0n, dtype=torch.float64, requires_grad=True)
    tgt = torch.tensor(pr.target, dtype=torch.float64)
    q, p = q0, p0
    for _ in range(T):
        gq, gp = torch.autograd.grad(H(q, p), (q, p), create_graph=True)
        q, p = q + gp / T, p - gq / T
    L = H(q0, p0) + lam * ((q - tgt) ** 2).sum()
    L.backward()
    r = oracle.shoot_gradient(pr.q0, p0n, pr.target, T, sigma, lam)
    assert abs(r["loss"] - L.item()) < 1e-12 * abs(L.item())
    assert rel(r["grad_p0"], p0.grad.numpy()) < 1e-10
    assert rel(r["grad_q0"], q0.grad.numpy()) < 1e-10


def test_golden_regression_fixture():
    # tests/golden/oracle_n8_T5.txt was written by tests/golden/make_golden.py
    # (oracle only); it guards against silent changes of the oracle.
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_n8_T5.txt")
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split("=", 1)
            vals[k.strip()] = np.array([float(x) for x in v.split()])
    q0 = vals["q0"].reshape(-1, 3); p0 = vals["p0"].reshape(-1, 3); t = vals["target"].reshape(-1, 3)
    r = oracle.shoot_gradient(q0, p0, t, 5, 0.3, 10.0)
    assert abs(r["loss"] - vals["loss"][0]) < 1e-12 * abs(vals["loss"][0])
    assert rel(r["grad_p0"], vals["grad_p0"].reshape(-1, 3)) < 1e-12
    assert rel(r["grad_q0"], vals["grad_q0"].reshape(-1, 3)) < 1e-12
    assert rel(r["q1"], vals["q1"].reshape(-1, 3)) < 1e-13


# ---------------------------------------------------------------- L-BFGS

def test_lbfgs_solves_convex_quadratic():
    # The minimiser of 1/2 x^T A x - b^T x is A^{-1} b (numpy solve).
    rng = np.random.default_rng(40)
    n = 30
    M = rng.normal(size=(n, n))
    A = M @ M.T + n * np.eye(n)
    b = rng.normal(size=n)
    # ||g|| <= 3e-9 ||g0||: much further and the line search meets the FP64
    # resolution of f for this problem
    r = oracle.lbfgs_quadratic(A, b, np.zeros(n), m=10, max_iter=200, grad_tol=3e-9)
    assert r["status"] == 0
    assert rel(r["x"], np.linalg.solve(A, b)) < 1e-8


def test_lbfgs_rosenbrock_reaches_ones():
    x0 = np.array([-1.2, 1.0] * 5)
    r = oracle.lbfgs_rosenbrock(x0, m=10, max_iter=1000, grad_tol=1e-9)
    assert r["status"] == 0
    assert np.abs(r["x"] - 1.0).max() < 1e-6


def test_register_decreases_loss_and_first_step_follows_gradient():
    pr = ls.ellipsoid_pair(64, seed=4, n_bumps=4)
    T, sigma, lam = 5, 0.25, 10.0
    r = oracle.register(pr.q0, pr.target, T, sigma, lam, max_iter=15, grad_tol=1e-8)
    tr = r["trace"]
    assert np.all(np.diff(tr) < 0)  # Armijo: every accepted step lowers the loss
    assert tr[-1] < 0.2 * tr[0]
    assert abs(oracle.loss(pr.q0, r["x"], pr.target, T, sigma, lam) - r["f"]) < 1e-12 * r["f"]
    # the first iterate lies on the ray p0 = -a g0 of the closed-form gradient
    r1 = oracle.register(pr.q0, pr.target, T, sigma, lam, max_iter=1, grad_tol=0.0)
    g0 = 2 * lam * dense_K(pr.q0, pr.q0, sigma) @ (pr.q0 - pr.target)
    a = -np.sum(r1["x"] * g0) / np.sum(g0 * g0)
    assert a > 0 and rel(r1["x"], -a * g0) < 1e-12
