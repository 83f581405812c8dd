"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances are normwise relative errors, ||x - x_ref|| / ||x_ref||:
1e-5 for StepForward / StepBackward outputs, q(1), p(1), H0 and the loss,
1e-4 for the gradients dL/dp0 and dL/dq0.  The kernels sum FP32 terms with
compensation and combine in double-single / FP64; the observed errors are
far below these bounds, and each test also prints them.
"""
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
    a = np.asarray(a, dtype=np.float64).ravel()
    b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(x):
    return torch.tensor(np.asarray(x, dtype=np.float32), device="cuda")


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def f32(x):
    """The FP32 values the kernels actually receive, in FP64 for the oracle."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def cloud(n, seed, radius=0.3, pscale=0.3):
    rng = np.random.default_rng(seed)
    return rng.uniform(-radius, radius, size=(n, 3)), rng.normal(0.0, pscale, size=(n, 3))


# ---------------------------------------------------------------- single steps

@pytest.mark.parametrize("n,sigma", [(1, 0.3), (2, 0.3), (7, 0.25), (64, 0.2), (65, 0.2),
                                     (1000, 0.1), (3001, 0.05), (4096, 0.1)])
def test_step_forward_parity(n, sigma):
    q, p = cloud(n, 100 + n)
    q, p = f32(q), f32(p)
    Hq, Hp = gs().step_forward(dev(q), dev(p), sigma)
    rq, rp = oracle.step_forward(q, p, sigma)
    eq, ep = rel(host(Hq), rq), rel(host(Hp), rp)
    print("N=%d step_forward rel err Hq %.2e Hp %.2e" % (n, eq, ep))
    assert ep < 1e-5
    assert eq < 1e-5 or np.linalg.norm(rq) < 1e-12


@pytest.mark.parametrize("n,sigma", [(1, 0.3), (5, 0.25), (64, 0.2), (127, 0.2), (1000, 0.1), (4096, 0.1)])
def test_step_backward_parity(n, sigma):
    q, p = cloud(n, 200 + n)
    rng = np.random.default_rng(300 + n)
    a, b = f32(rng.normal(size=(n, 3))), f32(rng.normal(size=(n, 3)))
    q, p = f32(q), f32(p)
    da, db = gs().step_backward(dev(q), dev(p), dev(a), dev(b), sigma)
    ra, rb = oracle.step_backward(q, p, a, b, sigma)
    ea, eb = rel(host(da), ra), rel(host(db), rb)
    print("N=%d step_backward rel err dalpha %.2e dbeta %.2e" % (n, ea, eb))
    assert eb < 1e-5
    assert ea < 1e-5 or np.linalg.norm(ra) < 1e-12


def test_step_host_and_device_pointers_agree_bitwise():
    q, p = cloud(777, 5)
    Hq_d, Hp_d = gs().step_forward(dev(q), dev(p), 0.1)
    Hq_h, Hp_h = gs().step_forward(np.float32(q), np.float32(p), 0.1)
    assert np.array_equal(host(Hq_d), Hq_h.astype(np.float64))
    assert np.array_equal(host(Hp_d), Hp_h.astype(np.float64))


# ---------------------------------------------------------------- forward flow

@pytest.mark.parametrize("n,T,sigma,pscale", [(256, 10, 0.2, 0.05), (1000, 7, 0.1, 0.02), (4096, 20, 0.1, 0.01)])
def test_shoot_forward_parity(n, T, sigma, pscale):
    pr = ls.ellipsoid_pair(n, seed=0, n_bumps=4 if n <= 256 else 8)
    q0 = f32(pr.q0)
    p0 = f32(ls.random_momentum(n, pscale, seed=1))
    q1, p1, H0 = gs().shoot_forward(dev(q0), dev(p0), T, sigma)
    rq1, rp1 = oracle.shoot_forward(q0, p0, T, sigma)
    rH0 = oracle.hamiltonian(q0, p0, sigma)
    e = (rel(host(q1), rq1), rel(host(p1), rp1), abs(H0 - rH0) / abs(rH0))
    print("N=%d T=%d shoot_forward rel err q1 %.2e p1 %.2e H0 %.2e" % ((n, T) + e))
    assert e[0] < 1e-5 and e[1] < 1e-5 and e[2] < 1e-5


def test_single_landmark_straight_line_gpu():
    q0 = np.array([[0.3, -1.2, 2.5]])
    p0 = np.array([[0.7, 0.1, -0.4]])
    q1, p1, H0 = gs().shoot_forward(dev(q0), dev(p0), 13, 0.37)
    assert np.allclose(host(p1), f32(p0), rtol=0, atol=1e-7)
    assert np.allclose(host(q1), f32(q0) + f32(p0), rtol=0, atol=1e-6)
    assert abs(H0 - 0.5 * float(np.sum(f32(p0) ** 2))) < 1e-7


def test_momentum_conserved_gpu():
    pr = ls.ellipsoid_pair(2000, seed=3)
    p0 = f32(ls.random_momentum(2000, 0.02, seed=4))
    _, p1, _ = gs().shoot_forward(dev(pr.q0), dev(p0), 20, 0.1)
    drift = np.abs(host(p1).sum(0) - p0.sum(0)).max()
    assert drift < 1e-5 * np.abs(p0).sum(0).max()


# ---------------------------------------------------------------- gradient

def _grad_case(n, T, sigma, lam, pscale, seed=0, bumps=8):
    pr = ls.ellipsoid_pair(n, seed=seed, n_bumps=bumps)
    q0, t = f32(pr.q0), f32(pr.target)
    p0 = f32(ls.random_momentum(n, pscale, seed=seed + 1)) if pscale > 0 else np.zeros_like(q0)
    return q0, p0, t


@pytest.mark.parametrize("n,T,sigma,lam,pscale", [
    (256, 10, 0.2, 10.0, 0.0),      # 256 landmarks, 4 bumps geometry, p0 = 0
    (256, 10, 0.2, 10.0, 0.05),
    (1, 5, 0.3, 10.0, 0.3),
    (333, 6, 0.15, 3.0, 0.03),      # ragged N
    (4096, 20, 0.1, 10.0, 0.01),    # the timed workload
])
def test_shoot_gradient_parity(n, T, sigma, lam, pscale):
    q0, p0, t = _grad_case(n, T, sigma, lam, pscale, bumps=4 if n <= 256 else 8)
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, lam)
    r = oracle.shoot_gradient(q0, p0, t, T, sigma, lam)
    e = (abs(loss - r["loss"]) / abs(r["loss"]), rel(host(gp), r["grad_p0"]), rel(host(gq), r["grad_q0"]))
    print("N=%d T=%d shoot_gradient rel err loss %.2e grad_p0 %.2e grad_q0 %.2e" % ((n, T) + e))
    assert e[0] < 1e-5
    assert e[1] < 1e-4
    assert e[2] < 1e-4


def test_gradient_closed_form_p0_zero_full_size_sampled():
    # 16384 landmarks, sigma = 0.05: at p0 = 0, dL/dp0 = 2 lambda K(q0)(q0 - t),
    # i.e. Hp(q0, q0 - t) row by row; checked on sampled rows by the oracle.
    n, T, sigma, lam = 16384, 40, 0.05, 10.0
    q0, p0, t = _grad_case(n, T, sigma, lam, 0.0)
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, lam)
    rows = np.random.default_rng(0).choice(n, size=64, replace=False)
    _, Hp = oracle.step_forward_rows(q0, q0 - t, sigma, rows)
    assert rel(host(gp)[rows], 2 * lam * Hp) < 1e-4
    assert rel(host(gq), 2 * lam * (q0 - t)) < 1e-5
    assert abs(loss - lam * np.sum((q0 - t) ** 2)) < 1e-5 * loss


def test_step_forward_full_size_sampled():
    n, sigma = 65536, 0.05
    pr = ls.ellipsoid_pair(n, seed=2)
    q = f32(pr.q0)
    p = f32(ls.random_momentum(n, 0.003, seed=3))
    Hq, Hp = gs().step_forward(dev(q), dev(p), sigma)
    rows = np.random.default_rng(1).choice(n, size=48, replace=False)
    rq, rp = oracle.step_forward_rows(q, p, sigma, rows)
    assert rel(host(Hp)[rows], rp) < 1e-5
    assert rel(host(Hq)[rows], rq) < 1e-5


def test_step_backward_full_size_sampled():
    # StepBackward at the largest size with non-zero adjoints (the dynamic
    # reverse sweep's pair sums), 48 sampled targets against the oracle.
    n, sigma = 65536, 0.05
    pr = ls.ellipsoid_pair(n, seed=4)
    q = f32(pr.q0)
    p = f32(ls.random_momentum(n, 0.003, seed=5))
    rng = np.random.default_rng(6)
    a, b = f32(rng.normal(0.0, 1.0, size=(n, 3))), f32(rng.normal(0.0, 0.01, size=(n, 3)))
    da, db = gs().step_backward(dev(q), dev(p), dev(a), dev(b), sigma)
    rows = np.random.default_rng(7).choice(n, size=48, replace=False)
    ra, rb = oracle.step_backward_rows(q, p, a, b, sigma, rows)
    ea, eb = rel(host(da)[rows], ra), rel(host(db)[rows], rb)
    print("N=%d step_backward 48 rows: dalpha %.2e dbeta %.2e" % (n, ea, eb))
    assert ea < 1e-5 and eb < 1e-5


def test_gradient_full_size_one_step():
    # The fused forward and reverse step kernels at 65536 landmarks with a
    # moving flow (p0 != 0), against the oracle's whole gradient (T = 1:
    # about 1.3e10 FP64 pair evaluations on the host).
    n, T, sigma, lam = 65536, 1, 0.05, 10.0
    pr = ls.ellipsoid_pair(n, seed=8)
    q0, t = f32(pr.q0), f32(pr.target)
    p0 = f32(ls.random_momentum(n, 0.003, seed=9))
    loss, gp, gq = gs().shoot_gradient(dev(q0), dev(p0), dev(t), T, sigma, lam)
    r = oracle.shoot_gradient(q0, p0, t, T, sigma, lam)
    e = (abs(loss - r["loss"]) / abs(r["loss"]), rel(host(gp), r["grad_p0"]), rel(host(gq), r["grad_q0"]))
    print("N=%d T=%d gradient rel err loss %.2e grad_p0 %.2e grad_q0 %.2e" % ((n, T) + e))
    assert e[0] < 1e-5 and e[1] < 1e-4 and e[2] < 1e-4


def test_gradient_deterministic_bitwise():
    q0, p0, t = _grad_case(1500, 8, 0.1, 10.0, 0.02)
    a = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 8, 0.1, 10.0)
    b = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 8, 0.1, 10.0)
    assert a[0] == b[0]
    assert torch.equal(a[1], b[1]) and torch.equal(a[2], b[2])


def test_gradient_host_pointers_match_device():
    q0, p0, t = _grad_case(500, 5, 0.2, 10.0, 0.05)
    a = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 5, 0.2, 10.0)
    b = gs().shoot_gradient(np.float32(q0), np.float32(p0), np.float32(t), 5, 0.2, 10.0)
    assert a[0] == b[0]
    assert np.array_equal(host(a[1]), b[1].astype(np.float64))


def test_interleaved_sizes_keep_padding_exact():
    # A larger problem followed by a smaller one must not leak stale state
    # into the padded landmarks.
    q0, p0, t = _grad_case(700, 5, 0.1, 10.0, 0.03)
    big = _grad_case(2100, 5, 0.1, 10.0, 0.03, seed=9)
    gs().shoot_gradient(dev(big[0]), dev(big[1]), dev(big[2]), 5, 0.1, 10.0)
    loss, gp, _ = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 5, 0.1, 10.0)
    r = oracle.shoot_gradient(q0, p0, t, 5, 0.1, 10.0)
    assert abs(loss - r["loss"]) < 1e-5 * r["loss"]
    assert rel(host(gp), r["grad_p0"]) < 1e-4


# ---------------------------------------------------------------- errors

def test_nonfinite_input_is_reported():
    q0, p0, t = _grad_case(100, 3, 0.2, 10.0, 0.05)
    p0 = p0.copy()
    p0[17, 1] = np.nan
    with pytest.raises(gs().GShootError) as ei:
        gs().shoot_gradient(dev(q0), dev(p0), dev(t), 3, 0.2, 10.0)
    assert ei.value.status == -5
    # the library stays usable
    q0, p0, t = _grad_case(100, 3, 0.2, 10.0, 0.05)
    loss, _, _ = gs().shoot_gradient(dev(q0), dev(p0), dev(t), 3, 0.2, 10.0)
    assert np.isfinite(loss)


def test_invalid_arguments_rejected():
    q = dev(np.zeros((4, 3)))
    with pytest.raises(gs().GShootError) as ei:
        gs().shoot_forward(q, q, 0, 0.1)
    assert ei.value.status == -1
    with pytest.raises(gs().GShootError):
        gs().shoot_forward(q, q, 5, -1.0)


def test_compensated_pair_sums_beat_sequential_fp32():
    # Section 2.2: accumulating the pair terms sequentially in FP32 loses
    # accuracy.  On the metric's workload (N = 4096, sigma = 0.1), the
    # kernel's compensated FP32 sums are compared with a plain sequential
    # FP32 accumulation of the same FP32 terms, both against the FP64 oracle,
    # for 64 sampled targets.
    pr = ls.ellipsoid_pair(4096, seed=0, n_bumps=8)
    q, p = f32(pr.q0), f32(ls.random_momentum(4096, 0.01, seed=1))
    sigma = 0.1
    rows = np.random.default_rng(3).choice(4096, size=64, replace=False)
    _, Hp = gs().step_forward(dev(q), dev(p), sigma)
    _, rp = oracle.step_forward_rows(q, p, sigma, rows)
    q32, p32 = q.astype(np.float32), p.astype(np.float32)
    seq = np.empty((rows.size, 3))
    for r, i in enumerate(rows):
        d = q32[i] - q32
        g = np.exp(-(d * d).sum(1, dtype=np.float32) / np.float32(2 * sigma * sigma)).astype(np.float32)
        terms = (g[:, None] * p32).astype(np.float32)
        seq[r] = np.add.accumulate(terms, axis=0, dtype=np.float32)[-1]  # left to right in FP32
    e_kernel = rel(host(Hp)[rows], rp)
    e_seq = rel(seq, rp)
    print("Hp of 64 targets: compensated kernel %.2e, sequential FP32 %.2e" % (e_kernel, e_seq))
    assert e_kernel < e_seq / 2
