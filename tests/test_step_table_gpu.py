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


def _ragged_variant_npad():
    """A padded count in [1024, 4096] whose table row gives the full-size
    CTAs (the RK4, terminal and planar kernels) clusters that do not divide
    the tile, forward and reverse; None if the table has none."""
    import os
    import re
    path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_1907_04839_gb300", "csrc", "step_table.inc")
    rows = [tuple(int(v) for v in m.group(1).split(","))
            for m in re.finditer(r"^\s*\{([0-9, ]+)\},\s*$", open(path).read(), re.M)]
    for r in rows:
        if 1024 <= r[0] <= 4096 and 128 % r[3] and 64 % r[6]:
            return r[0]
    return None


@pytest.mark.parametrize("dim", [3, 2])
@pytest.mark.parametrize("integrator,h_at", [("rk4", "start"), ("euler", "end"), ("rk4", "end")])
def test_variant_kernels_with_clusters_that_do_not_divide_the_tile(dim, integrator, h_at):
    """The RK4, terminal and planar kernels in the table's uneven cluster
    sizes (chosen from the table, so the check survives a regenerated one)."""
    import math
    import paper_1907_04839_gb300 as gsh
    npad = _ragged_variant_npad()
    if npad is None:
        pytest.skip("the table gives the variant kernels no cluster that leaves the tile unevenly split")
    n, T = npad - 5, 4
    if dim == 3:
        sigma = 0.1
        pr = ls.ellipsoid_pair(n, seed=13, n_bumps=8)
        q0 = pr.q0.astype(np.float32).astype(np.float64)
        t = pr.target.astype(np.float32).astype(np.float64)
        p0 = ls.random_momentum(n, 0.03, seed=14).astype(np.float32).astype(np.float64)
    else:
        # smooth planar momenta (the displacement over the kernel's row mass), as
        # in the planar tests: random ones make the planar flow ill-conditioned
        sigma = 0.05
        pr = ls.ellipse_pair(n, seed=13, n_bumps=8)
        perimeter = 2 * math.pi * math.sqrt((1.0 ** 2 + 0.6 ** 2) / 2)
        mass = max(1.0, math.sqrt(2 * math.pi) * sigma * n / perimeter)
        q0 = pr.q0.astype(np.float32).astype(np.float64)
        t = pr.target.astype(np.float32).astype(np.float64)
        p0 = ((pr.target - pr.q0) / mass).astype(np.float32).astype(np.float64)
    d = lambda x: torch.tensor(x.astype(np.float32), device="cuda")
    loss, gp, gq = gsh.shoot_gradient(d(q0), d(p0), d(t), T, sigma, 10.0, integrator=integrator, h_at=h_at)
    r = oracle.shoot_gradient_v(q0, p0, t, T, sigma, 10.0, integrator, h_at)
    el = abs(loss - r["loss"]) / abs(r["loss"])
    ep, eq = rel(gp.cpu().numpy(), r["grad_p0"]), rel(gq.cpu().numpy(), r["grad_q0"])
    print("%d-D %s/%s N=%d: loss %.2e grad_p0 %.2e grad_q0 %.2e" % (dim, integrator, h_at, n, el, ep, eq))
    assert el < 1e-5 and ep < 1e-4 and eq < 1e-4
