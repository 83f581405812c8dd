"""Writes tests/golden/oracle_n8_T5.txt from the FP64 oracle alone.

A regression fixture: eight landmarks, T = 5, sigma = 0.3, lambda = 10, with a
random initial momentum.  The values come only from ``oracle`` (the loss of
Eq. 3 and its gradient by the reverse sweep of Algorithm 1); nothing from the
CUDA path.  Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402


def main():
    rng = np.random.default_rng(2024)
    q0 = rng.uniform(-0.3, 0.3, size=(8, 3))
    p0 = rng.normal(0.0, 0.3, size=(8, 3))
    t = q0 + rng.normal(0.0, 0.1, size=(8, 3))
    r = oracle.shoot_gradient(q0, p0, t, 5, 0.3, 10.0)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_n8_T5.txt")

    def fmt(a):
        return " ".join("%.17g" % x for x in np.ravel(a))

    with open(out, "w") as f:
        f.write("# FP64 oracle regression fixture: N=8, T=5, sigma=0.3, lambda=10\n")
        f.write("# loss of Eq. 3 and its gradient (reverse sweep of Algorithm 1)\n")
        f.write("# written by tests/golden/make_golden.py (oracle only)\n")
        for k, v in (("q0", q0), ("p0", p0), ("target", t), ("loss", [r["loss"]]),
                     ("grad_p0", r["grad_p0"]), ("grad_q0", r["grad_q0"]), ("q1", r["q1"]),
                     ("p1", r["p1"])):
            f.write("%s = %s\n" % (k, fmt(v)))


if __name__ == "__main__":
    main()
