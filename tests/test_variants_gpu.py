"""The variants of the discretisation on the GPU against the FP64 oracle:
RK4 steps with their exact adjoint, and the loss with the kinetic term at
t = 1.  Tolerances as for the plain method: 1e-5 normwise relative on q(1),
p(1) and the loss, 1e-4 on the gradients."""
import numpy as np
import pytest

import landmark_synth as ls
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

VARIANTS = [("rk4", "start"), ("euler", "end"), ("rk4", "end")]


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


def problem(n, seed, pscale=0.03):
    pr = ls.ellipsoid_pair(n, seed=seed, n_bumps=8 if n > 300 else 4)
    return f32(pr.q0), f32(ls.random_momentum(n, pscale, seed=seed + 1)), f32(pr.target)


@pytest.mark.parametrize("n,T,sigma", [(1, 3, 0.3), (300, 6, 0.2), (2001, 5, 0.1), (4096, 3, 0.1)])
def test_rk4_forward_matches_oracle(n, T, sigma):
    q0, p0, _ = problem(n, 5)
    q1, p1, H0 = gs().shoot_forward(dev(q0), dev(p0), T, sigma, integrator="rk4")
    rq, rp = oracle.shoot_forward_v(q0, p0, T, sigma, "rk4")
    eq, ep = rel(q1.cpu().numpy(), rq), rel(p1.cpu().numpy(), rp)
    eh = abs(H0 - oracle.hamiltonian(q0, p0, sigma)) / oracle.hamiltonian(q0, p0, sigma)
    print("RK4 N=%d T=%d: q1 %.2e p1 %.2e H0 %.2e" % (n, T, eq, ep, eh))
    assert eq < 1e-5 and ep < 1e-5 and eh < 1e-5


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
@pytest.mark.parametrize("n,T,sigma", [(1, 4, 0.3), (257, 6, 0.2), (1500, 4, 0.1)])
def test_variant_gradient_matches_oracle(integrator, h_at, n, T, sigma):
    q0, p0, t = problem(n, 7)
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, 10.0, integrator=integrator, h_at=h_at)
    r = oracle.shoot_gradient_v(q0, p0, t, T, sigma, 10.0, integrator, h_at)
    el = abs(loss - r["loss"]) / abs(r["loss"])
    ep, eq = rel(gp.cpu().numpy(), r["grad_p0"]), rel(gq.cpu().numpy(), r["grad_q0"])
    print("%s/%s N=%d: loss %.2e grad_p0 %.2e grad_q0 %.2e" % (integrator, h_at, n, el, ep, eq))
    assert el < 1e-5 and ep < 1e-4 and eq < 1e-4


def test_rk4_kinetic_end_gradient_at_4096_landmarks():
    q0, p0, t = problem(4096, 9, pscale=0.01)
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 3, 0.1, 10.0, integrator="rk4", h_at="end")
    r = oracle.shoot_gradient_v(q0, p0, t, 3, 0.1, 10.0, "rk4", "end")
    assert abs(loss - r["loss"]) < 1e-5 * abs(r["loss"])
    assert rel(gp.cpu().numpy(), r["grad_p0"]) < 1e-4 and rel(gq.cpu().numpy(), r["grad_q0"]) < 1e-4


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
def test_variant_checkpointing_is_bitwise_identical(integrator, h_at):
    # T = 9 with k = 4: segments of 4, 4 and 1 steps.
    q0, p0, t = problem(1000, 11)
    a = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 9, 0.1, 10.0, integrator=integrator, h_at=h_at)
    b = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 9, 0.1, 10.0, ckpt_every=4, integrator=integrator, h_at=h_at)
    assert a[0] == b[0]
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


@pytest.mark.parametrize("integrator,h_at", VARIANTS)
def test_variant_closed_form_at_zero_momentum(integrator, h_at):
    q0, _, t = problem(700, 13)
    lam, sigma = 10.0, 0.1
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(np.zeros_like(q0)), dev(t), 5, sigma, lam, integrator=integrator,
                                       h_at=h_at)
    resid = q0 - t
    K = np.exp(-((q0[:, None, :] - q0[None, :, :]) ** 2).sum(-1) / (2 * sigma ** 2))
    assert abs(loss - lam * np.sum(resid ** 2)) < 1e-5 * loss
    assert rel(gp.cpu().numpy(), 2 * lam * K @ resid) < 1e-4
    assert rel(gq.cpu().numpy(), 2 * lam * resid) < 1e-4


def test_euler_start_variant_is_the_plain_path():
    q0, p0, t = problem(800, 15)
    a = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 6, 0.1, 10.0)
    b = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 6, 0.1, 10.0, integrator="euler", h_at="start")
    assert a[0] == b[0] and torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


@pytest.mark.parametrize("integrator,h_at", [("rk4", "start"), ("rk4", "end")])
def test_variant_register_first_iterates_match_oracle(integrator, h_at):
    pr = ls.ellipsoid_pair(256, seed=17, n_bumps=4)
    q0, t = f32(pr.q0), f32(pr.target)
    p0, info = gs().register(q0, t, 5, 0.2, 10.0, max_iter=3, grad_tol=0.0, integrator=integrator, h_at=h_at)
    r = oracle.register_v(q0, t, 5, 0.2, 10.0, integrator, h_at, max_iter=3, grad_tol=0.0)
    e = rel(p0, r["x"])
    print("%s/%s register: p0 rel err %.2e loss %.9g / %.9g" % (integrator, h_at, e, info["loss"], r["f"]))
    assert info["iters"] == 3 and info["evals"] == r["evals"]
    assert e < 1e-4 and abs(info["loss"] - r["f"]) < 1e-5 * r["f"]


def test_autograd_function_carries_the_variant():
    q0, p0, t = problem(300, 19)
    q = dev(q0).requires_grad_(True)
    p = dev(p0).requires_grad_(True)
    L = gs().shoot(q, p, dev(t), 4, 0.2, 10.0, integrator="rk4", h_at="end")
    L.backward()
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 4, 0.2, 10.0, integrator="rk4", h_at="end")
    assert L.item() == loss
    assert torch.equal(p.grad, gp) and torch.equal(q.grad, gq)


def test_flow_points_rejects_rk4():
    q0, p0, _ = problem(50, 21)
    with pytest.raises(gs().GShootError) as ei:
        import ctypes
        lib = gs().load()
        prm = gs()._params(50, 4, 0.2, integrator="rk4")
        x = dev(q0)
        out = torch.empty_like(x)
        gs().check(lib.flow_points(ctypes.byref(prm), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(dev(p0).data_ptr()),
                                   50, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(out.data_ptr()), None))
    assert ei.value.status == -1


def test_rk4_kinetic_end_gradient_at_16384_landmarks():
    # Full-size check of the variant kernels in the launch configuration of
    # large problems (several waves, load-balancing cluster scheduling).
    q0, p0, t = problem(16384, 23, pscale=0.01)
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 2, 0.05, 10.0, integrator="rk4", h_at="end")
    r = oracle.shoot_gradient_v(q0, p0, t, 2, 0.05, 10.0, "rk4", "end")
    el, ep, eq = abs(loss - r["loss"]) / abs(r["loss"]), rel(gp.cpu().numpy(), r["grad_p0"]), rel(gq.cpu().numpy(),
                                                                                                     r["grad_q0"])
    print("rk4/end N=16384: loss %.2e grad_p0 %.2e grad_q0 %.2e" % (el, ep, eq))
    assert el < 1e-5 and ep < 1e-4 and eq < 1e-4
