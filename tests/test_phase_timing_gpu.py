"""Phase events inside the gradient graph (gs_set_phase_timing): they time
the forward and the reverse sweep of the replayed graph and change nothing
in its results."""
import ctypes

import numpy as np
import pytest

import landmark_synth as ls

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def test_phase_events_time_both_sweeps_and_leave_results_unchanged():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    n, T = 2048, 12
    pr = ls.ellipsoid_pair(n, seed=3, n_bumps=8)
    p0 = ls.random_momentum(n, 0.01, seed=4)
    dev = torch.device("cuda", 0)
    dq, dp, dt = (torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(dev) for a in (pr.q0, p0, pr.target))
    prm = gsh.GsParams(N=n, T=T, ckpt_every=0, sigma=0.1, lambda_=10.0, lbfgs_m=10, max_iter=10, grad_tol=1e-5)
    P = lambda x: ctypes.c_void_p(x.data_ptr())
    sp = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)

    def grad():
        g = torch.empty((n, 3), dtype=torch.float32, device=dev)
        loss = ctypes.c_double(0.0)
        gsh.check(lib.shoot_gradient(ctypes.byref(prm), P(dq), P(dp), P(dt), ctypes.byref(loss), P(g), None, sp))
        return g.cpu().numpy(), loss.value

    g0, l0 = grad()
    gsh.check(lib.gs_set_phase_timing(1))
    try:
        grad()  # capture the timed graph
        stream = torch.cuda.current_stream(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g1, l1 = grad()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        f, b = ctypes.c_double(0.0), ctypes.c_double(0.0)
        gsh.check(lib.gs_phase_times(ctypes.byref(f), ctypes.byref(b)))
    finally:
        gsh.check(lib.gs_set_phase_timing(0))
    outer = e0.elapsed_time(e1)
    print("phase times: forward %.4f ms, reverse %.4f ms, whole call %.4f ms" % (f.value, b.value, outer))
    assert np.array_equal(g0, g1) and l0 == l1
    assert f.value > 0.0 and b.value > 0.0
    # both sweeps lie inside the call
    assert f.value + b.value <= outer * 1.001 + 1e-3
