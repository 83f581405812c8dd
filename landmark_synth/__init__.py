"""Seeded synthetic landmark workloads.

This module only draws inputs.  It holds none of the shooting method's
arithmetic and is imported by both the FP64 oracle's tests and the CUDA path's
tests and benchmarks, so that both sides see byte-identical inputs.

The paper's data (1847 Poisson-disk landmarks on a medial-temporal-lobe
template mesh, registered to 34 subjects, Section 3.1) is not available.  The
stand-in keeps the shape of that work: a smooth closed 3-D surface sampled
roughly uniformly (template), and a smoothly deformed copy of it (target).

Recipe (fixed draw order, one ``numpy.random.default_rng(seed)`` stream):

1. template: ``n`` points area-uniform on the ellipsoid with semi-axes
   ``axes``.  A direction u is drawn uniformly on the unit sphere and mapped to
   x = (a u1, b u2, c u3); it is kept with probability
   ||(u1/a, u2/b, u3/c)|| * min(a, b, c), which is the ratio of the ellipsoid's
   area element to the sphere's, normalised to at most one.  Proposals are
   drawn in batches until ``n`` are accepted.
2. jitter: iid N(0, jitter^2) per coordinate, added to the template.
3. bump centres: ``n_bumps`` distinct template indices drawn uniformly.
4. bump amplitudes: iid N(0, amp^2) per coordinate, one 3-vector per bump.
5. target = template + sum_b A_b exp(-||x - c_b||^2 / (2 sigma_b^2)).

Planar landmarks (the paper codes the 2-D case too): ``ellipse_pair`` draws
``n`` points arc-length-uniform on the ellipse with semi-axes ``axes`` (an
angle t uniform in [0, 2 pi), kept with probability
sqrt(a^2 sin^2 t + b^2 cos^2 t) / max(a, b)), then jitter, bump centres and
amplitudes and the target exactly as in steps 2-5, in two dimensions.

Population (one template, many subjects; the shape of Section 3.1's study of
34 subjects with 1847 landmarks each): a base surface is drawn by steps 1-2
from ``default_rng(seed)``.  Subject s draws steps 3-5 from its own stream
``default_rng((seed, s))`` on the base surface.  The template is the mean of
the subjects, as the paper builds its template by averaging the (rigidly
aligned) subject landmark sets; the synthetic subjects need no alignment.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "LandmarkPair",
    "ellipsoid_pair",
    "random_momentum",
    "batched_requests",
    "poisson_trace",
    "Population",
    "population",
    "ellipse_pair",
]


@dataclasses.dataclass
class LandmarkPair:
    q0: np.ndarray       # (N, 3) float64 template landmarks
    target: np.ndarray   # (N, 3) float64 target landmarks
    seed: int

    @property
    def n(self) -> int:
        return int(self.q0.shape[0])

    def as_f32(self):
        return (np.ascontiguousarray(self.q0, dtype=np.float32),
                np.ascontiguousarray(self.target, dtype=np.float32))


def _ellipsoid_surface(rng: np.random.Generator, n: int, axes) -> np.ndarray:
    a, b, c = (float(x) for x in axes)
    m = min(a, b, c)
    out = []
    have = 0
    while have < n:
        batch = max(64, 2 * (n - have))
        u = rng.standard_normal((batch, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        w = np.sqrt((u[:, 0] / a) ** 2 + (u[:, 1] / b) ** 2 + (u[:, 2] / c) ** 2) * m
        keep = rng.random(batch) < w
        x = u[keep] * np.array([a, b, c])
        out.append(x)
        have += x.shape[0]
    return np.concatenate(out, axis=0)[:n]


def ellipsoid_pair(n: int, seed: int = 0, n_bumps: int = 8,
                   axes=(1.0, 0.8, 0.6), jitter: float = 0.01,
                   bump_sigma: float = 0.3, bump_amp: float = 0.1) -> LandmarkPair:
    """Template on an ellipsoid surface and a bump-deformed target (see module doc)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    x = _ellipsoid_surface(rng, n, axes)
    x = x + rng.normal(0.0, jitter, size=x.shape)
    nb = min(n_bumps, n)
    centres = x[rng.choice(n, size=nb, replace=False)]
    amps = rng.normal(0.0, bump_amp, size=(nb, 3))
    disp = np.zeros_like(x)
    for cb, ab in zip(centres, amps):
        w = np.exp(-np.sum((x - cb) ** 2, axis=1) / (2.0 * bump_sigma ** 2))
        disp += w[:, None] * ab[None, :]
    return LandmarkPair(q0=np.ascontiguousarray(x), target=np.ascontiguousarray(x + disp), seed=seed)


def random_momentum(n: int, scale: float, seed: int) -> np.ndarray:
    """iid N(0, scale^2) initial momenta, (N, 3) float64."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, size=(n, 3))


def batched_requests(count: int = 512, n_lo: int = 500, n_hi: int = 8000,
                     sigmas=(0.05, 0.1, 0.2), first_seed: int = 1, trace_seed: int = 0):
    """Independent registration problems: N log-uniform in [n_lo, n_hi],
    sigma uniform over ``sigmas``, each with its own generator seed.
    Returns a list of dicts {seed, n, sigma}."""
    rng = np.random.default_rng(trace_seed)
    logn = rng.uniform(math.log(n_lo), math.log(n_hi), size=count)
    ns = np.clip(np.round(np.exp(logn)).astype(int), n_lo, n_hi)
    sig = rng.choice(np.asarray(sigmas, dtype=float), size=count)
    return [dict(seed=first_seed + k, n=int(ns[k]), sigma=float(sig[k])) for k in range(count)]


def poisson_trace(count: int, rate: float, n_lo: int = 1000, n_hi: int = 50000,
                  trace_seed: int = 0, first_seed: int = 1):
    """Poisson arrival trace: exponential inter-arrival gaps with mean 1/rate
    seconds, N log-uniform in [n_lo, n_hi].  Returns a list of dicts
    {seed, n, t_arrival}."""
    rng = np.random.default_rng(trace_seed)
    gaps = rng.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    logn = rng.uniform(math.log(n_lo), math.log(n_hi), size=count)
    ns = np.clip(np.round(np.exp(logn)).astype(int), n_lo, n_hi)
    return [dict(seed=first_seed + k, n=int(ns[k]), t_arrival=float(t[k])) for k in range(count)]


@dataclasses.dataclass
class Population:
    template: np.ndarray  # (N, 3) float64: the mean of the subjects
    targets: list         # per subject (N, 3) float64
    seed: int

    @property
    def n(self) -> int:
        return int(self.template.shape[0])


def population(n: int = 1847, subjects: int = 34, seed: int = 0, n_bumps: int = 8,
               axes=(1.0, 0.8, 0.6), jitter: float = 0.01,
               bump_sigma: float = 0.3, bump_amp: float = 0.1) -> Population:
    """One template and `subjects` targets with corresponding landmarks (see
    the module doc)."""
    if n < 1 or subjects < 1:
        raise ValueError("n and subjects must be >= 1")
    rng = np.random.default_rng(seed)
    base = _ellipsoid_surface(rng, n, axes)
    base = base + rng.normal(0.0, jitter, size=base.shape)
    nb = min(n_bumps, n)
    targets = []
    for s in range(subjects):
        r = np.random.default_rng((seed, s))
        centres = base[r.choice(n, size=nb, replace=False)]
        amps = r.normal(0.0, bump_amp, size=(nb, 3))
        disp = np.zeros_like(base)
        for cb, ab in zip(centres, amps):
            w = np.exp(-np.sum((base - cb) ** 2, axis=1) / (2.0 * bump_sigma ** 2))
            disp += w[:, None] * ab[None, :]
        targets.append(np.ascontiguousarray(base + disp))
    template = np.ascontiguousarray(np.mean(np.stack(targets), axis=0))
    return Population(template=template, targets=targets, seed=seed)


def ellipse_pair(n: int, seed: int = 0, n_bumps: int = 8, axes=(1.0, 0.6), jitter: float = 0.01,
                 bump_sigma: float = 0.3, bump_amp: float = 0.1) -> LandmarkPair:
    """Planar template on an ellipse and a bump-deformed target (module doc)."""
    if n < 1:
        raise ValueError("n must be >= 1")
    rng = np.random.default_rng(seed)
    a, b = (float(x) for x in axes)
    out, have = [], 0
    while have < n:
        batch = max(64, 2 * (n - have))
        t = rng.uniform(0.0, 2.0 * math.pi, size=batch)
        w = np.sqrt((a * np.sin(t)) ** 2 + (b * np.cos(t)) ** 2) / max(a, b)
        keep = rng.random(batch) < w
        out.append(np.stack([a * np.cos(t[keep]), b * np.sin(t[keep])], axis=1))
        have += int(keep.sum())
    x = np.concatenate(out, axis=0)[:n]
    x = x + rng.normal(0.0, jitter, size=x.shape)
    nb = min(n_bumps, n)
    centres = x[rng.choice(n, size=nb, replace=False)]
    amps = rng.normal(0.0, bump_amp, size=(nb, 2))
    disp = np.zeros_like(x)
    for cb, ab in zip(centres, amps):
        wgt = np.exp(-np.sum((x - cb) ** 2, axis=1) / (2.0 * bump_sigma ** 2))
        disp += wgt[:, None] * ab[None, :]
    return LandmarkPair(q0=np.ascontiguousarray(x), target=np.ascontiguousarray(x + disp), seed=seed)
