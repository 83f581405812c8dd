"""Every compiled variant of the fused time-step kernels against the FP64
oracle.  A variant is (threads per CTA, targets per thread, warp groups that
split each CTA's sources) plus a cluster size; gs_set_step_config forces it
for both sweeps.  Sizes are ragged so that tiles, source splits, chunks and
warp-group pieces all end short."""
import ctypes

import numpy as np
import pytest

import landmark_synth as ls
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FWD = [(64, 1, 1), (64, 2, 1), (64, 4, 1), (128, 1, 1), (128, 2, 1), (128, 4, 1), (256, 1, 1), (256, 2, 1),
       (64, 1, 2), (128, 1, 2), (128, 1, 4), (256, 1, 4)]
BWD = [(32, 1, 1), (64, 1, 1), (64, 2, 1), (128, 1, 1), (128, 2, 1), (256, 1, 1), (64, 1, 2), (128, 1, 2),
       (128, 1, 4), (256, 1, 4)]


def rel(a, b):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def case():
    n, T, sigma, lam = 1000, 4, 0.12, 10.0
    pr = ls.ellipsoid_pair(n, seed=5, n_bumps=8)
    q0 = pr.q0.astype(np.float32).astype(np.float64)
    t = pr.target.astype(np.float32).astype(np.float64)
    p0 = ls.random_momentum(n, 0.02, seed=6).astype(np.float32).astype(np.float64)
    ref = oracle.shoot_gradient(q0, p0, t, T, sigma, lam)
    return n, T, sigma, lam, q0, p0, t, ref


def _run(case, fwd, bwd, cluster_f, cluster_b):
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    n, T, sigma, lam, q0, p0, t, ref = case
    gsh.check(lib.gs_set_step_config(0, fwd[0], fwd[1], fwd[2], cluster_f))
    gsh.check(lib.gs_set_step_config(1, bwd[0], bwd[1], bwd[2], cluster_b))
    try:
        d = lambda x: torch.tensor(x.astype(np.float32), device="cuda")
        loss, gp, gq = gsh.shoot_gradient(d(q0), d(p0), d(t), T, sigma, lam)
    finally:
        gsh.check(lib.gs_set_step_config(0, 0, 0, 0, 0))
        gsh.check(lib.gs_set_step_config(1, 0, 0, 0, 0))
    e = (abs(loss - ref["loss"]) / abs(ref["loss"]), rel(gp.cpu().numpy(), ref["grad_p0"]),
         rel(gq.cpu().numpy(), ref["grad_q0"]))
    return e


@pytest.mark.parametrize("fwd", FWD)
def test_forward_variants(case, fwd):
    for c in (4, 16):
        if c > fwd[0] // fwd[2] * fwd[1]:
            continue
        e = _run(case, fwd, (64, 1, 1), c, 8)
        print("fwd %s c=%d: loss %.2e grad_p0 %.2e grad_q0 %.2e" % ((fwd, c) + e))
        assert e[0] < 1e-5 and e[1] < 1e-4 and e[2] < 1e-4


@pytest.mark.parametrize("bwd", BWD)
def test_reverse_variants(case, bwd):
    for c in (4, 16):
        if c > bwd[0] // bwd[2] * bwd[1]:
            continue
        e = _run(case, (128, 1, 1), bwd, 16, c)
        print("bwd %s c=%d: loss %.2e grad_p0 %.2e grad_q0 %.2e" % ((bwd, c) + e))
        assert e[0] < 1e-5 and e[1] < 1e-4 and e[2] < 1e-4


@pytest.mark.parametrize("c", [3, 6, 10, 12, 14])
def test_clusters_that_do_not_divide_the_tile(case, c):
    """Cluster sizes that are not powers of two: the last CTA of each cluster
    reduces fewer targets than the others.  The CTA shapes the step table
    uses, forward and reverse alike."""
    for fwd, bwd in (((128, 1, 1), (64, 1, 1)), ((64, 1, 1), (32, 1, 1))):
        e = _run(case, fwd, bwd, c, c)
        print("fwd %s bwd %s c=%d: loss %.2e grad_p0 %.2e grad_q0 %.2e" % ((fwd, bwd, c) + e))
        assert e[0] < 1e-5 and e[1] < 1e-4 and e[2] < 1e-4


def test_cluster_size_outside_1_to_16_is_rejected():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    for c in (0, 17, 32):
        assert lib.gs_set_step_config(0, 64, 1, 1, c) == -1
        assert lib.gs_set_step_config(1, 32, 1, 1, c) == -1


def test_unknown_variant_is_rejected():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    assert lib.gs_set_step_config(0, 96, 1, 1, 8) == -1
    assert lib.gs_set_step_config(1, 64, 1, 3, 8) == -1
