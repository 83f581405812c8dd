"""Failure detection on the GPU without a fault: a device wait that nothing
completes ends at the library's iteration limit, the call reports
GS_ETIMEOUT (-4), and the context stays usable for the next call."""
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


@pytest.mark.parametrize("which", [0, 1])
def test_expired_wait_reports_timeout_and_the_context_survives(which):
    lib = gs().load()
    secs = ctypes.c_double(0.0)
    st = lib.gs_check_wait_timeout(which, ctypes.byref(secs), None)
    print("wait %d: status %d after %.3f s (%s)" % (which, st, secs.value, lib.gs_last_error().decode()))
    assert st == -4
    assert secs.value < 30.0
    # The next call runs normally and is correct.
    pr = ls.ellipsoid_pair(300, seed=2, n_bumps=4)
    q0 = pr.q0.astype(np.float32)
    t = pr.target.astype(np.float32)
    p0 = ls.random_momentum(300, 0.03, seed=3).astype(np.float32)
    d = lambda a: torch.tensor(a, device="cuda")
    loss, gp, gq = gs().shoot_gradient(d(q0), d(p0), d(t), 6, 0.2, 10.0)
    r = oracle.shoot_gradient(q0.astype(np.float64), p0.astype(np.float64), t.astype(np.float64), 6, 0.2, 10.0)
    assert abs(loss - r["loss"]) < 1e-5 * r["loss"]
    e = np.linalg.norm(gp.cpu().numpy() - r["grad_p0"]) / np.linalg.norm(r["grad_p0"])
    assert e < 1e-4
