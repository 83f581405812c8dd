"""The per-step combine of split partials in FP64 against the double-single
default (gs_set_combine_precision).  Both must match the FP64 oracle within
the C-13 tolerances; each error is printed, and the two results agree to
far below the tolerances."""
import numpy as np
import pytest

import landmark_synth as ls
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n,T,sigma", [(1000, 7, 0.1), (4096, 20, 0.1)])
def test_fp64_and_double_single_combine_match_oracle(n, T, sigma):
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    pr = ls.ellipsoid_pair(n, seed=21, n_bumps=8)
    q0 = pr.q0.astype(np.float32).astype(np.float64)
    t = pr.target.astype(np.float32).astype(np.float64)
    p0 = ls.random_momentum(n, 0.01, seed=22).astype(np.float32).astype(np.float64)
    ref = oracle.shoot_gradient(q0, p0, t, T, sigma, 10.0)
    d = lambda x: torch.tensor(x.astype(np.float32), device="cuda")
    out = {}
    try:
        for f64 in (0, 1):
            gsh.check(lib.gs_set_combine_precision(f64))
            loss, gp, gq = gsh.shoot_gradient(d(q0), d(p0), d(t), T, sigma, 10.0)
            q1, p1, h0 = gsh.shoot_forward(d(q0), d(p0), T, sigma)
            out[f64] = (loss, gp.cpu().numpy(), gq.cpu().numpy(), q1.cpu().numpy(), p1.cpu().numpy())
    finally:
        gsh.check(lib.gs_set_combine_precision(0))
    for f64, (loss, gp, gq, q1, p1) in out.items():
        e = (abs(loss - ref["loss"]) / abs(ref["loss"]), rel(gp, ref["grad_p0"]), rel(gq, ref["grad_q0"]),
             rel(q1, ref["q1"]), rel(p1, ref["p1"]))
        print("N=%d %s combine: loss %.2e grad_p0 %.2e grad_q0 %.2e q1 %.2e p1 %.2e"
              % ((n, "FP64" if f64 else "double-single") + e))
        assert e[0] < 1e-5 and e[1] < 1e-4 and e[2] < 1e-4 and e[3] < 1e-5 and e[4] < 1e-5
    assert rel(out[1][1], out[0][1]) < 1e-6


def test_fp64_combine_in_batched_registration():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    probs = []
    for k, (n, sigma) in enumerate(((600, 0.1), (1300, 0.2))):
        pr = ls.ellipsoid_pair(n, seed=30 + k, n_bumps=8)
        probs.append(dict(q0=pr.q0.astype(np.float32), target=pr.target.astype(np.float32), sigma=sigma, lam=10.0))
    try:
        gsh.check(lib.gs_set_combine_precision(1))
        res = gsh.register_batch(probs, T=5, max_iter=3, grad_tol=0.0)
    finally:
        gsh.check(lib.gs_set_combine_precision(0))
    for pr, (p, info) in zip(probs, res):
        r = oracle.register(pr["q0"].astype(np.float64), pr["target"].astype(np.float64), 5, pr["sigma"],
                            10.0, max_iter=3, grad_tol=0.0)
        print("batched FP64 combine N=%d: p0 rel err %.2e" % (pr["q0"].shape[0], rel(p, r["x"])))
        assert rel(p, r["x"]) < 1e-4
