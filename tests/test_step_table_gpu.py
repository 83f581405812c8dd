"""The measured step-configuration table against the size rule it refines.
At sizes where the table picks another CTA or cluster size than the rule
(and at one where the two agree), the gradient with the table and without it
both match the FP64 oracle, and agree with each other to rounding."""
import numpy as np
import pytest

import landmark_synth as ls
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("n", [300, 3011, 4096, 7100])
def test_table_and_rule_both_match_oracle(n):
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    T, sigma, lam = 4, 0.1, 10.0
    pr = ls.ellipsoid_pair(n, seed=11, n_bumps=8)
    q0 = pr.q0.astype(np.float32).astype(np.float64)
    t = pr.target.astype(np.float32).astype(np.float64)
    p0 = ls.random_momentum(n, 0.01, seed=12).astype(np.float32).astype(np.float64)
    ref = oracle.shoot_gradient(q0, p0, t, T, sigma, lam)
    d = lambda x: torch.tensor(x.astype(np.float32), device="cuda")
    out = {}
    try:
        for on in (1, 0):
            gsh.check(lib.gs_set_step_table(on))
            loss, gp, gq = gsh.shoot_gradient(d(q0), d(p0), d(t), T, sigma, lam)
            out[on] = (loss, gp.cpu().numpy(), gq.cpu().numpy())
    finally:
        gsh.check(lib.gs_set_step_table(1))
    for on, (loss, gp, gq) in out.items():
        assert abs(loss - ref["loss"]) / abs(ref["loss"]) < 1e-5, on
        assert rel(gp, ref["grad_p0"]) < 1e-4, on
        assert rel(gq, ref["grad_q0"]) < 1e-4, on
    assert rel(out[1][1], out[0][1]) < 1e-5
