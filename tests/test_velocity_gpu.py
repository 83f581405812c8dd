"""The Eq. 4 velocity field and points carried through the deformation
(velocity_field, flow_points) against the FP64 oracle.  Tolerance: 1e-5
normwise relative, as for q(1) and p(1)."""
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


def f32(x):
    return np.asarray(x, np.float32).astype(np.float64)


def dev(x):
    return torch.tensor(np.asarray(x, np.float32), device="cuda")


def state(n, seed, pscale=0.05):
    pr = ls.ellipsoid_pair(n, seed=seed, n_bumps=8)
    return f32(pr.q0), f32(ls.random_momentum(n, pscale, seed=seed + 1))


def points(m, seed, radius=1.1):
    return f32(np.random.default_rng(seed).uniform(-radius, radius, size=(m, 3)))


@pytest.mark.parametrize("n,m,sigma", [(1, 1, 0.3), (100, 57, 0.2), (1000, 3001, 0.1), (4096, 777, 0.1),
                                       (333, 129, 0.05)])
def test_velocity_field_parity(n, m, sigma):
    q, p = state(n, 3)
    x = points(m, 4)
    v = gs().velocity_field(dev(q), dev(p), dev(x), sigma)
    r = oracle.velocity(x, q, p, sigma)
    e = rel(v.cpu().numpy(), r)
    print("N=%d M=%d velocity rel err %.2e" % (n, m, e))
    assert e < 1e-5


def test_velocity_at_landmarks_is_hp():
    q, p = state(500, 5)
    v = gs().velocity_field(dev(q), dev(p), dev(q), 0.1)
    _, Hp = oracle.step_forward(q, p, 0.1)
    assert rel(v.cpu().numpy(), Hp) < 1e-5


@pytest.mark.parametrize("n,m,T,sigma", [(500, 333, 7, 0.1), (4096, 1000, 20, 0.1), (1, 5, 4, 0.3)])
def test_flow_points_parity(n, m, T, sigma):
    # The parity bar applies to a well-conditioned flow: first check that the
    # oracle's own result moves by much less than the tolerance when p0 is
    # perturbed by 1e-7 relative.  (With random momenta ten times larger the
    # flow at N = 4096 is chaotic and amplifies such a perturbation to 0.8.)
    q, p = state(n, 7, pscale=0.02)
    x = points(m, 8)
    x1 = gs().flow_points(dev(q), dev(p), dev(x), T, sigma)
    r = oracle.flow_points(q, p, x, T, sigma)
    assert rel(oracle.flow_points(q, p * (1 + 1e-7), x, T, sigma), r) < 1e-6
    e = rel(x1.cpu().numpy(), r)
    disp = rel(x1.cpu().numpy() - x, r - x)
    print("N=%d M=%d T=%d flow_points rel err %.2e (displacement %.2e)" % (n, m, T, e, disp))
    assert e < 1e-5
    assert disp < 1e-4


def test_flow_points_landmarks_follow_q():
    q, p = state(2000, 9, pscale=0.02)
    x1 = gs().flow_points(dev(q), dev(p), dev(q), 10, 0.1)
    q1, _, _ = gs().shoot_forward(dev(q), dev(p), 10, 0.1)
    assert rel(x1.cpu().numpy(), q1.cpu().numpy()) < 1e-6


def test_flow_points_far_points_stay():
    q, p = state(300, 11)
    x = np.array([[80.0, 0.0, 0.0], [0.0, -60.0, 7.0]])
    x1 = gs().flow_points(dev(q), dev(p), dev(x), 6, 0.1)
    assert np.array_equal(x1.cpu().numpy(), x.astype(np.float32))


def test_host_and_device_points_agree_bitwise():
    q, p = state(700, 13)
    x = points(450, 14)
    v_dev = gs().velocity_field(dev(q), dev(p), dev(x), 0.1).cpu().numpy()
    v_host = gs().velocity_field(q.astype(np.float32), p.astype(np.float32), x.astype(np.float32), 0.1)
    assert np.array_equal(v_dev, v_host)
    x1_dev = gs().flow_points(dev(q), dev(p), dev(x), 5, 0.1).cpu().numpy()
    x1_host = gs().flow_points(q.astype(np.float32), p.astype(np.float32), x.astype(np.float32), 5, 0.1)
    assert np.array_equal(x1_dev, x1_host)


def test_point_errors():
    q, p = state(64, 15)
    x = points(10, 16).astype(np.float32)
    x[3, 1] = np.nan
    with pytest.raises(gs().GShootError) as ei:
        gs().velocity_field(q.astype(np.float32), p.astype(np.float32), x, 0.1)
    assert ei.value.status == -5
    with pytest.raises(gs().GShootError) as ei:
        gs().flow_points(q.astype(np.float32), p.astype(np.float32), x, 4, 0.1)
    assert ei.value.status == -5
    import ctypes
    lib = gs().load()
    assert lib.velocity_field(64, 0, 0.1, None, None, None, None, None) == -1
