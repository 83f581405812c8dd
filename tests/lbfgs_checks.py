"""Checks of an L-BFGS run from its iterates alone (Section 2.1's optimiser
with the settings the library states: memory m, initial scaling
gamma = s.y / y.y, strong Wolfe with c1 = 1e-4 and c2 = 0.9, first direction
-g, a pair kept only if s.y > 1e-12 ||s|| ||y||).

Given iterates x_0 .. x_K of a run and a function returning (f, g) at any
point, each step s_k = x_{k+1} - x_k must

* start downhill: g_k . s_k < 0;
* satisfy the strong Wolfe conditions for the step it took:
  f_{k+1} <= f_k + c1 g_k . s_k and |g_{k+1} . s_k| <= c2 |g_k . s_k|;
* point along -H_k g_k, where H_k is the BFGS inverse update of gamma I,
  applied as a dense matrix over the last m kept pairs, oldest first.

None of this uses the optimiser's code: the dense update is a different
computation from the two-loop recursion, and the Wolfe test needs only the
accepted points.  `fg` supplies the (f, g) values the checks use."""
import numpy as np


def dense_direction(g, pairs, m):
    n = g.size
    use = pairs[-m:]
    if not use:
        return -g
    s_l, y_l = use[-1]
    H = (s_l @ y_l) / (y_l @ y_l) * np.eye(n)
    for s, y in use:
        rho = 1.0 / (s @ y)
        V = np.eye(n) - rho * np.outer(y, s)
        H = V.T @ H @ V + rho * np.outer(s, s)
    return -H @ g


def check_iterates(xs, fg, m=10, c1=1e-4, c2=0.9, f_slack=1e-9, wolfe_slack=1e-3, cos_tol=1e-5):
    """Assert the three properties above for every step of xs; returns the
    per-step records (for printing)."""
    vals = [fg(x) for x in xs]
    pairs, out = [], []
    for k in range(len(xs) - 1):
        x0, x1 = xs[k].ravel(), xs[k + 1].ravel()
        f0, g0 = vals[k][0], vals[k][1].ravel()
        f1, g1 = vals[k + 1][0], vals[k + 1][1].ravel()
        s, y = x1 - x0, g1 - g0
        slope = float(g0 @ s)
        d = dense_direction(g0, pairs, m)
        cos = float(s @ d / (np.linalg.norm(s) * np.linalg.norm(d)))
        rec = dict(k=k, f0=f0, f1=f1, slope=slope, curv=float(g1 @ s), cos=cos)
        out.append(rec)
        assert slope < 0.0, rec
        assert f1 <= f0 + c1 * slope + f_slack * abs(f0), ("sufficient decrease", rec)
        assert abs(float(g1 @ s)) <= c2 * abs(slope) * (1.0 + wolfe_slack), ("curvature", rec)
        assert cos >= 1.0 - cos_tol, ("direction", rec)
        if s @ y > 1e-12 * np.linalg.norm(s) * np.linalg.norm(y):
            pairs.append((s, y))
    return out
