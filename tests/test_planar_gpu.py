"""Planar (2-D) landmarks on the GPU against the FP64 oracle: the forward
flow, the gradient of every variant of the discretisation, checkpointing
and register.  Tolerances as in 3-D: 1e-5 normwise relative on q(1), p(1)
and the loss, 1e-4 on the gradients."""
import math

import numpy as np
import pytest

import landmark_synth as ls
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VARIANTS = [("euler", "start"), ("rk4", "start"), ("euler", "end"), ("rk4", "end")]


def gs():
    import paper_1907_04839_gb300 as m
    return m


def rel(a, b):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def dev(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda")


def problem(n, seed, sigma):
    """Planar landmarks on an ellipse and smooth momenta: the displacement to
    the target divided by the kernel's row mass (about sqrt(2 pi) sigma n /
    perimeter), a field like a registration's.  Random momenta at these
    kernel widths make the planar flow ill-conditioned: the FP32 rounding of
    the inputs alone would move p(1) by more than the tolerance."""
    pr = ls.ellipse_pair(n, seed=seed, n_bumps=8 if n > 300 else 4)
    perimeter = 2 * math.pi * math.sqrt((1.0 ** 2 + 0.6 ** 2) / 2)
    mass = max(1.0, math.sqrt(2 * math.pi) * sigma * n / perimeter)
    return f32(pr.q0), f32((pr.target - pr.q0) / mass), f32(pr.target)


@pytest.mark.parametrize("integrator", ["euler", "rk4"])
@pytest.mark.parametrize("n,T,sigma", [(1, 3, 0.3), (333, 8, 0.1), (2049, 5, 0.05), (4096, 4, 0.05)])
def test_planar_forward_matches_oracle(integrator, n, T, sigma):
    q0, p0, _ = problem(n, 3, sigma)
    q1, p1, H0 = gs().shoot_forward(dev(q0), dev(p0), T, sigma, integrator=integrator)
    assert tuple(q1.shape) == (n, 2)
    rq, rp = oracle.shoot_forward_v(q0, p0, T, sigma, integrator)
    h = oracle.hamiltonian_d(q0, p0, sigma)
    eq, ep, eh = rel(q1.cpu().numpy(), rq), rel(p1.cpu().numpy(), rp), abs(H0 - h) / h
    print("2-D %s N=%d: q1 %.2e p1 %.2e H0 %.2e" % (integrator, n, eq, ep, eh))
    assert eq < 1e-5 and ep < 1e-5 and eh < 1e-5


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
@pytest.mark.parametrize("n,T,sigma", [(1, 4, 0.3), (500, 6, 0.1), (3000, 4, 0.05)])
def test_planar_gradient_matches_oracle(integrator, h_at, n, T, sigma):
    q0, p0, t = problem(n, 5, sigma)
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, 10.0, integrator=integrator, h_at=h_at)
    r = oracle.shoot_gradient_v(q0, p0, t, T, sigma, 10.0, integrator, h_at)
    el = abs(loss - r["loss"]) / abs(r["loss"])
    ep, eq = rel(gp.cpu().numpy(), r["grad_p0"]), rel(gq.cpu().numpy(), r["grad_q0"])
    print("2-D %s/%s N=%d: loss %.2e grad_p0 %.2e grad_q0 %.2e" % (integrator, h_at, n, el, ep, eq))
    assert el < 1e-5 and ep < 1e-4 and eq < 1e-4


@pytest.mark.parametrize("integrator,h_at", [("euler", "start"), ("rk4", "end")])
def test_planar_checkpointing_is_bitwise_identical(integrator, h_at):
    q0, p0, t = problem(1200, 7, 0.05)
    a = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 9, 0.05, 10.0, integrator=integrator, h_at=h_at)
    b = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 9, 0.05, 10.0, ckpt_every=4, integrator=integrator, h_at=h_at)
    assert a[0] == b[0] and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def test_planar_and_3d_calls_interleave_on_one_workspace():
    # The same N in 2-D and 3-D in turn: the padded records must be clean each time.
    q0, p0, t = problem(777, 9, 0.1)
    pr = ls.ellipsoid_pair(777, seed=9, n_bumps=4)
    q3, t3 = f32(pr.q0), f32(pr.target)
    p3 = f32(ls.random_momentum(777, 0.03, seed=10))
    for _ in range(2):
        l2, g2, _ = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 5, 0.1, 10.0)
        l3, g3, _ = gs().shoot_gradient(dev(q3), dev(p3), dev(t3), 5, 0.1, 10.0)
        r2 = oracle.shoot_gradient_v(q0, p0, t, 5, 0.1, 10.0)
        r3 = oracle.shoot_gradient(q3, p3, t3, 5, 0.1, 10.0)
        assert rel(g2.cpu().numpy(), r2["grad_p0"]) < 1e-4 and rel(g3.cpu().numpy(), r3["grad_p0"]) < 1e-4


def test_planar_register_first_iterates_match_oracle():
    pr = ls.ellipse_pair(400, seed=11, n_bumps=4)
    q0, t = f32(pr.q0), f32(pr.target)
    p0, info = gs().register(q0, t, 6, 0.1, 10.0, max_iter=3, grad_tol=0.0)
    assert p0.shape == (400, 2)
    r = oracle.register_v(q0, t, 6, 0.1, 10.0, max_iter=3, grad_tol=0.0)
    e = rel(p0, r["x"])
    print("2-D register: p0 rel err %.2e loss %.9g / %.9g" % (e, info["loss"], r["f"]))
    assert info["iters"] == 3 and info["evals"] == r["evals"]
    assert e < 1e-4 and abs(info["loss"] - r["f"]) < 1e-5 * r["f"]
    d = np.linalg.norm(oracle.shoot_forward_v(q0, r["x"], 6, 0.1)[0] - t, axis=1)
    assert abs(info["avg_dist"] - d.mean()) < 1e-4 * d.mean()


def test_planar_equals_the_embedded_3d_problem():
    # Zero third coordinates add exact zeros to every sum.
    q0, p0, t = problem(600, 13, 0.1)
    z = lambda x: np.concatenate([x, np.zeros((x.shape[0], 1))], axis=1)
    l2, g2, h2 = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 5, 0.1, 10.0)
    l3, g3, h3 = gs().shoot_gradient(dev(z(q0)), dev(z(p0)), dev(z(t)), 5, 0.1, 10.0)
    assert abs(l2 - l3) <= 1e-6 * l3
    assert rel(g2.cpu().numpy(), g3.cpu().numpy()[:, :2]) < 1e-6
    assert float(g3[:, 2].abs().max()) == 0.0


@pytest.mark.parametrize("integrator,h_at", [("euler", "start"), ("rk4", "end")])
def test_planar_host_arrays_equal_device_arrays(integrator, h_at):
    # numpy inputs are staged through the workspace; the results are bitwise
    # those of device inputs.
    q0, p0, t = problem(900, 17, 0.1)
    ld, gpd, gqd = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 5, 0.1, 10.0, integrator=integrator, h_at=h_at)
    f = lambda a: np.asarray(a, np.float32)
    lh, gph, gqh = gs().shoot_gradient(f(q0), f(p0), f(t), 5, 0.1, 10.0, integrator=integrator, h_at=h_at)
    assert isinstance(gph, np.ndarray) and gph.shape == (900, 2)
    assert lh == ld
    assert np.array_equal(gph, gpd.cpu().numpy()) and np.array_equal(gqh, gqd.cpu().numpy())
