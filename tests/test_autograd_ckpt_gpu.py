"""Trajectory checkpointing of the reverse sweep and the torch autograd
Function: 16384 landmarks (sigma = 0.05, T = 40) checked against the oracle
gradient and central finite differences along random directions, then
65536 landmarks with the state checkpointed every 8 steps."""
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


def dev(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda")


def problem(n, seed=0, pscale=0.0):
    pr = ls.ellipsoid_pair(n, seed=seed, n_bumps=8)
    p0 = ls.random_momentum(n, pscale, seed=seed + 1) if pscale > 0 else np.zeros((n, 3))
    return pr.q0.astype(np.float32), p0.astype(np.float32), pr.target.astype(np.float32)


@pytest.mark.parametrize("T,k", [(10, 1), (10, 3), (10, 4), (10, 9), (7, 2)])
def test_checkpointing_is_bitwise_identical(T, k):
    q0, p0, t = problem(1500, pscale=0.02)
    a = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, 0.1, 10.0)
    b = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, 0.1, 10.0, ckpt_every=k)
    assert a[0] == b[0]
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def test_autograd_function_matches_library_gradient():
    q0, p0, t = problem(777, pscale=0.03)
    qd = dev(q0).requires_grad_(True)
    pd = dev(p0).requires_grad_(True)
    L = gs().shoot(qd, pd, dev(t), 6, 0.15, 10.0)
    assert L.dtype == torch.float64 and L.dim() == 0
    (2.5 * L).backward()
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 6, 0.15, 10.0)
    assert abs(L.item() - loss) == 0.0
    assert torch.allclose(pd.grad, 2.5 * gp, rtol=1e-6, atol=0)
    assert torch.allclose(qd.grad, 2.5 * gq, rtol=1e-6, atol=0)


def test_autograd_16384_vs_oracle_and_finite_differences():
    n, T, sigma, lam = 16384, 40, 0.05, 10.0
    q0, p0, t = problem(n, seed=5, pscale=0.002)
    qd = dev(q0).requires_grad_(True)
    pd = dev(p0).requires_grad_(True)
    L = gs().shoot(qd, pd, dev(t), T, sigma, lam)
    L.backward()
    gp = pd.grad.cpu().numpy().astype(np.float64)
    gq = qd.grad.cpu().numpy().astype(np.float64)
    r = oracle.shoot_gradient(q0.astype(np.float64), p0.astype(np.float64), t.astype(np.float64), T, sigma, lam)
    e = (abs(L.item() - r["loss"]) / r["loss"], rel(gp, r["grad_p0"]), rel(gq, r["grad_q0"]))
    print("N=16384 T=40 rel err loss %.2e grad_p0 %.2e grad_q0 %.2e" % e)
    assert e[0] < 1e-5 and e[1] < 1e-4 and e[2] < 1e-4
    # Central differences along 32 random unit directions.  The loss is
    # reduced in FP64 but carries the rounding noise of the FP32 pair sums.
    # That noise is measured as the scatter of the loss around its
    # first-order prediction at 8 tiny perturbations, and it sets the
    # tolerance at h = 1e-4.  The wider h = 1e-2 gives a tight check.
    rng = np.random.default_rng(11)
    f = lambda p: gs().shoot_gradient(dev(q0), dev(p), dev(t), T, sigma, lam)[0]
    L0 = L.item()
    resid = []
    for _ in range(8):
        u = rng.normal(size=p0.shape); u /= np.linalg.norm(u)
        pu = (p0 + 1e-6 * u).astype(np.float32).astype(np.float64)
        resid.append(f(pu) - (L0 + float(np.sum(gp * (pu - p0)))))
    dL = float(np.std(resid)) + 1e-14 * L0
    worst = {1e-4: 0.0, 1e-2: 0.0}
    for _ in range(32):
        v = rng.normal(size=p0.shape); v /= np.linalg.norm(v)
        an = float(np.sum(gp * v))
        for h in (1e-4, 1e-2):
            pp = (p0 + h * v).astype(np.float32).astype(np.float64)
            pm = (p0 - h * v).astype(np.float32).astype(np.float64)
            step = float(np.sum((pp - pm) * v)) / 2  # step after FP32 rounding of the inputs
            fd = (f(pp) - f(pm)) / (2 * step)
            dev_ = abs(fd - an)
            noise = 4 * np.sqrt(2) * dL / (2 * step)
            tol = noise + (2e-3 if h == 1e-4 else 1e-4) * abs(an)
            worst[h] = max(worst[h], dev_ / tol)
            assert dev_ <= tol, (h, fd, an, tol)
    print("loss noise %.2e; worst deviation / tolerance: h=1e-4 %.2f, h=1e-2 %.2f" % (dL, worst[1e-4], worst[1e-2]))


def test_checkpointed_65536_bitwise_and_closed_form():
    n, T, sigma, lam = 65536, 40, 0.05, 10.0
    q0, p0, t = problem(n, seed=7, pscale=0.001)
    a = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, lam)
    b = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, lam, ckpt_every=8)
    assert a[0] == b[0]
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])
    # at p0 = 0 the checkpointed gradient has the closed form 2 lambda K (q0 - t)
    z = np.zeros_like(p0)
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(z), dev(t), T, sigma, lam, ckpt_every=8)
    rows = np.random.default_rng(3).choice(n, size=32, replace=False)
    _, Hp = oracle.step_forward_rows(q0.astype(np.float64), (q0 - t).astype(np.float64), sigma, rows)
    assert rel(gp.cpu().numpy()[rows], 2 * lam * Hp) < 1e-4
