"""Persistent sweeps: one launch walks all T time steps of the forward (or
reverse) Euler sweep, its clusters meeting at a grid-wide barrier between
steps.  Each step is computed by the same configuration as the one-launch-
per-step kernels, so results must be bitwise identical to those (sweep
mode 0), and within the C-13 tolerances of the FP64 oracle."""
import ctypes

import numpy as np
import pytest

import landmark_synth as ls
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def gs():
    import paper_1907_04839_gb300 as m
    return m


def lib():
    return gs().load()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device="cuda")


def persistent(kind, n):
    out = ctypes.c_int32(-1)
    gs()._lib.check(lib().gs_sweep_persistent(kind, n, ctypes.byref(out)))
    return out.value


def set_mode(mode):
    gs()._lib.check(lib().gs_set_sweep_mode(mode))


def workload(n, seed=0, pscale=0.01):
    pr = ls.ellipsoid_pair(n, seed=seed, n_bumps=8 if n > 256 else 4)
    p0 = ls.random_momentum(n, pscale, seed=seed + 1)
    return (np.asarray(pr.q0, np.float32), np.asarray(p0, np.float32), np.asarray(pr.target, np.float32))


def grad_both_modes(q0, p0, t, T, sigma, lam):
    out = {}
    try:
        for mode in (-1, 0):
            set_mode(mode)
            loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, lam)
            out[mode] = (loss, gp.cpu().numpy(), gq.cpu().numpy())
    finally:
        set_mode(-1)
    return out


# Up to 4096 landmarks both sweeps fit on a GB300 at once; at 6000 the
# reverse sweep's shape (32-thread CTAs in clusters of 16) does not, so the
# persistent forward sweep is followed by per-step reverse launches.
@pytest.mark.parametrize("n,T,sigma,both", [(256, 10, 0.2, True), (1000, 7, 0.1, True), (2113, 20, 0.1, True),
                                            (4096, 20, 0.1, True), (6000, 5, 0.05, False)])
def test_sweep_gradient_bitwise_equal_to_per_step_launches(n, T, sigma, both):
    q0, p0, t = workload(n)
    fwd, bwd = persistent(0, n), persistent(1, n)
    print("N=%d persistent forward %d reverse %d" % (n, fwd, bwd))
    if both:
        assert fwd == 1 and bwd == 1, "the sweeps should fit on the device at this size"
    r = grad_both_modes(q0, p0, t, T, sigma, 10.0)
    assert r[-1][0] == r[0][0]
    assert np.array_equal(r[-1][1], r[0][1])
    assert np.array_equal(r[-1][2], r[0][2])


@pytest.mark.parametrize("n,T,sigma", [(1, 4, 0.2), (65, 6, 0.2), (1000, 7, 0.1), (4096, 20, 0.1)])
def test_sweep_gradient_matches_oracle(n, T, sigma):
    q0, p0, t = workload(n, seed=3, pscale=0.05)
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, 10.0)
    r = oracle.shoot_gradient(q0.astype(np.float64), p0.astype(np.float64), t.astype(np.float64), T, sigma, 10.0)
    e_l = abs(loss - r["loss"]) / abs(r["loss"])
    e_p, e_q = rel(gp.cpu().numpy(), r["grad_p0"]), rel(gq.cpu().numpy(), r["grad_q0"])
    print("N=%d T=%d loss %.2e grad_p0 %.2e grad_q0 %.2e" % (n, T, e_l, e_p, e_q))
    assert e_l < 1e-5 and e_p < 1e-4 and e_q < 1e-4


@pytest.mark.parametrize("n,T", [(300, 9), (4096, 20)])
def test_sweep_forward_bitwise_and_oracle(n, T):
    q0, p0, _ = workload(n, seed=5, pscale=0.05)
    out = {}
    try:
        for mode in (-1, 0):
            set_mode(mode)
            q1, p1, h0 = gs().shoot_forward(dev(q0), dev(p0), T, 0.1)
            out[mode] = (q1.cpu().numpy(), p1.cpu().numpy(), h0)
    finally:
        set_mode(-1)
    assert np.array_equal(out[-1][0], out[0][0]) and np.array_equal(out[-1][1], out[0][1])
    assert out[-1][2] == out[0][2]
    q1, p1 = oracle.shoot_forward(q0.astype(np.float64), p0.astype(np.float64), T, 0.1)
    h0 = oracle.hamiltonian(q0.astype(np.float64), p0.astype(np.float64), 0.1)
    assert rel(out[-1][0], q1) < 1e-5 and rel(out[-1][1], p1) < 1e-5
    assert abs(out[-1][2] - h0) / abs(h0) < 1e-5


def test_sweep_register_iterates_bitwise_equal():
    q0, _, t = workload(256)
    res = {}
    try:
        for mode in (-1, 0):
            set_mode(mode)
            p, info = gs().register(dev(q0), dev(t), 10, 0.2, 10.0, max_iter=5, grad_tol=0.0)
            res[mode] = (p.cpu().numpy(), info)
    finally:
        set_mode(-1)
    assert np.array_equal(res[-1][0], res[0][0])
    assert res[-1][1]["loss"] == res[0][1]["loss"]


def test_sweep_repeated_calls_are_bitwise_identical():
    # The barrier counters restart at every launch, and the copy ring's
    # phases run on across steps: repeated graphs must agree bit for bit.
    q0, p0, t = workload(4096)
    a = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 20, 0.1, 10.0)
    for _ in range(3):
        b = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 20, 0.1, 10.0)
        assert a[0] == b[0] and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
