"""The seeded input generators (CPU): determinism, shapes, and the
population's template being the mean of its subjects."""
import numpy as np

import landmark_synth as ls


def test_population_template_is_the_subject_mean_and_draws_are_seeded():
    a = ls.population(300, 6, seed=5)
    b = ls.population(300, 6, seed=5)
    assert a.n == 300 and len(a.targets) == 6
    for x, y in zip(a.targets, b.targets):
        assert np.array_equal(x, y)
    assert np.allclose(a.template, np.mean(np.stack(a.targets), axis=0), rtol=0, atol=1e-15)
    # subjects differ from each other and from the template
    assert min(np.abs(a.targets[0] - t).max() for t in a.targets[1:]) > 1e-3
    assert np.abs(a.targets[0] - a.template).max() > 1e-3
    c = ls.population(300, 6, seed=6)
    assert np.abs(c.template - a.template).max() > 1e-3


def test_ellipsoid_pair_is_seeded_and_on_the_surface_before_jitter():
    p = ls.ellipsoid_pair(2000, seed=9, n_bumps=4, jitter=0.0)
    q = ls.ellipsoid_pair(2000, seed=9, n_bumps=4, jitter=0.0)
    assert np.array_equal(p.q0, q.q0) and np.array_equal(p.target, q.target)
    r = (p.q0[:, 0] / 1.0) ** 2 + (p.q0[:, 1] / 0.8) ** 2 + (p.q0[:, 2] / 0.6) ** 2
    assert np.allclose(r, 1.0, atol=1e-12)


def test_ellipse_pair_is_seeded_planar_and_on_the_curve_before_jitter():
    p = ls.ellipse_pair(1500, seed=4, n_bumps=4, jitter=0.0)
    q = ls.ellipse_pair(1500, seed=4, n_bumps=4, jitter=0.0)
    assert p.q0.shape == (1500, 2) and np.array_equal(p.q0, q.q0) and np.array_equal(p.target, q.target)
    assert np.allclose((p.q0[:, 0] / 1.0) ** 2 + (p.q0[:, 1] / 0.6) ** 2, 1.0, atol=1e-12)
