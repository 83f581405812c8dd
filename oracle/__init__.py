"""FP64 CPU oracle for landmark geodesic shooting -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does.

The arithmetic lives in ``oracle.c`` (plain double loops, OpenMP over target
landmarks).  This module compiles it with gcc on first use (or via
:func:`build`) and exposes numpy-in / numpy-out wrappers.  Arrays are (N, 3)
float64, row-major.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
# objective callback of orc_lbfgs: f(ctx, x, g) returns f(x), writes the gradient
_FG = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_void_p, _D, _D)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP, no FMA contraction so
    that x86 and Arm hosts round identically)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-Wall", "-Wextra", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, cint, cd = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.orc_set_threads.argtypes = [cint]
            lib.orc_max_threads.restype = cint
            lib.orc_step_forward.argtypes = [i64, cd, _D, _D, _D, _D]
            lib.orc_step_backward.argtypes = [i64, cd, _D, _D, _D, _D, _D, _D]
            lib.orc_hamiltonian.argtypes = [i64, cd, _D, _D]
            lib.orc_hamiltonian.restype = cd
            lib.orc_shoot_forward.argtypes = [i64, cint, cd, _D, _D, _D, _D, _D, _D]
            lib.orc_loss.argtypes = [i64, cint, cd, cd, _D, _D, _D]
            lib.orc_loss.restype = cd
            lib.orc_shoot_gradient.argtypes = [i64, cint, cd, cd, _D, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_shoot_gradient.restype = cd
            lib.orc_velocity.argtypes = [i64, _D, i64, _D, _D, cd, _D]
            lib.orc_flow_points.argtypes = [i64, cint, cd, _D, _D, i64, _D, _D]
            _I = ctypes.POINTER(ctypes.c_int64)
            IP = ctypes.POINTER(ctypes.c_int)
            lib.orc_lbfgs_quadratic.argtypes = [i64, _D, _D, _D, cint, cint, cd, _D, IP, IP]
            lib.orc_lbfgs_quadratic.restype = cint
            lib.orc_lbfgs_rosenbrock.argtypes = [i64, _D, cint, cint, cd, _D, IP, IP]
            lib.orc_lbfgs_rosenbrock.restype = cint
            lib.orc_lbfgs.argtypes = [i64, _D, _FG, ctypes.c_void_p, cint, cint, cd, _D, IP, IP, _D]
            lib.orc_lbfgs.restype = cint
            lib.orc_register.argtypes = [i64, cint, cd, cd, cint, cint, cd, _D, _D, _D, _D, IP, IP, _D]
            lib.orc_register.restype = cint
            lib.orc_shoot_forward_v.argtypes = [cint, i64, cint, cd, cint, _D, _D, _D, _D]
            lib.orc_step_forward_d.argtypes = [cint, i64, cd, _D, _D, _D, _D]
            lib.orc_step_backward_d.argtypes = [cint, i64, cd, _D, _D, _D, _D, _D, _D]
            lib.orc_hamiltonian_d.argtypes = [cint, i64, cd, _D, _D]
            lib.orc_hamiltonian_d.restype = cd
            lib.orc_loss_v.argtypes = [cint, i64, cint, cd, cd, cint, cint, _D, _D, _D]
            lib.orc_loss_v.restype = cd
            lib.orc_shoot_gradient_v.argtypes = [cint, i64, cint, cd, cd, cint, cint, _D, _D, _D, _D, _D, _D, _D, _D]
            lib.orc_shoot_gradient_v.restype = cd
            lib.orc_register_v.argtypes = [cint, i64, cint, cd, cd, cint, cint, cint, cint, cd, _D, _D, _D, _D, IP,
                                           IP, _D]
            lib.orc_register_v.restype = cint
            lib.orc_step_forward_rows.argtypes = [i64, cd, _D, _D, i64, _I, _D, _D]
            lib.orc_step_backward_rows.argtypes = [i64, cd, _D, _D, _D, _D, i64, _I, _D, _D]
            _lib = lib
    return _lib


def _in(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 3 or (n is not None and a.shape[0] != n):
        raise ValueError("expected an (N, 3) array, got shape %r" % (a.shape,))
    return a


def _p(a):
    return a.ctypes.data_as(_D) if a is not None else None


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def max_threads() -> int:
    return int(_load().orc_max_threads())


def step_forward(q, p, sigma):
    """StepForward: returns (Hq, Hp) of Eq. 2 at (q, p)."""
    q = _in(q); n = q.shape[0]; p = _in(p, n)
    Hq = np.empty_like(q); Hp = np.empty_like(q)
    _load().orc_step_forward(n, float(sigma), _p(q), _p(p), _p(Hq), _p(Hp))
    return Hq, Hp


def step_backward(q, p, alpha, beta, sigma):
    """StepBackward: returns (dalpha, dbeta), the adjoint pair sums."""
    q = _in(q); n = q.shape[0]
    p, alpha, beta = _in(p, n), _in(alpha, n), _in(beta, n)
    da = np.empty_like(q); db = np.empty_like(q)
    _load().orc_step_backward(n, float(sigma), _p(q), _p(p), _p(alpha), _p(beta), _p(da), _p(db))
    return da, db


def _rows(rows):
    r = np.ascontiguousarray(rows, dtype=np.int64)
    return r, r.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def step_forward_rows(q, p, sigma, rows):
    """StepForward for the target landmarks ``rows`` only: (Hq, Hp), (m, 3)."""
    q = _in(q); n = q.shape[0]; p = _in(p, n)
    r, rp = _rows(rows)
    if r.size and (r.min() < 0 or r.max() >= n):
        raise IndexError("row index out of range")
    Hq = np.empty((r.size, 3)); Hp = np.empty((r.size, 3))
    _load().orc_step_forward_rows(n, float(sigma), _p(q), _p(p), r.size, rp, _p(Hq), _p(Hp))
    return Hq, Hp


def step_backward_rows(q, p, alpha, beta, sigma, rows):
    """StepBackward for the target landmarks ``rows`` only: (dalpha, dbeta)."""
    q = _in(q); n = q.shape[0]
    p, alpha, beta = _in(p, n), _in(alpha, n), _in(beta, n)
    r, rp = _rows(rows)
    if r.size and (r.min() < 0 or r.max() >= n):
        raise IndexError("row index out of range")
    da = np.empty((r.size, 3)); db = np.empty((r.size, 3))
    _load().orc_step_backward_rows(n, float(sigma), _p(q), _p(p), _p(alpha), _p(beta), r.size, rp,
                                   _p(da), _p(db))
    return da, db


def hamiltonian(q, p, sigma) -> float:
    q = _in(q); p = _in(p, q.shape[0])
    return float(_load().orc_hamiltonian(q.shape[0], float(sigma), _p(q), _p(p)))


def shoot_forward(q0, p0, T, sigma, trajectory=False):
    """Forward flow; returns (q1, p1) or (q1, p1, traj_q, traj_p) with
    trajectories shaped (T+1, N, 3)."""
    q0 = _in(q0); n = q0.shape[0]; p0 = _in(p0, n)
    q1 = np.empty_like(q0); p1 = np.empty_like(q0)
    tq = tp = None
    if trajectory:
        tq = np.empty((T + 1, n, 3)); tp = np.empty((T + 1, n, 3))
    _load().orc_shoot_forward(n, int(T), float(sigma), _p(q0), _p(p0), _p(q1), _p(p1), _p(tq), _p(tp))
    return (q1, p1, tq, tp) if trajectory else (q1, p1)


def loss(q0, p0, target, T, sigma, lam) -> float:
    q0 = _in(q0); n = q0.shape[0]
    p0, target = _in(p0, n), _in(target, n)
    return float(_load().orc_loss(n, int(T), float(sigma), float(lam), _p(q0), _p(p0), _p(target)))


def shoot_gradient(q0, p0, target, T, sigma, lam):
    """ComputeGradient: returns dict(loss, grad_p0, grad_q0, q1, p1, H0)."""
    q0 = _in(q0); n = q0.shape[0]
    p0, target = _in(p0, n), _in(target, n)
    gp = np.empty_like(q0); gq = np.empty_like(q0)
    q1 = np.empty_like(q0); p1 = np.empty_like(q0)
    h0 = ctypes.c_double(0.0)
    L = _load().orc_shoot_gradient(n, int(T), float(sigma), float(lam), _p(q0), _p(p0), _p(target),
                                   _p(gp), _p(gq), _p(q1), _p(p1), ctypes.byref(h0))
    return dict(loss=float(L), grad_p0=gp, grad_q0=gq, q1=q1, p1=p1, H0=float(h0.value))


def velocity(x, q, p, sigma):
    """Eq. 4 velocity field at query points x (M, 3)."""
    x = _in(x); q = _in(q); p = _in(p, q.shape[0])
    v = np.empty_like(x)
    _load().orc_velocity(x.shape[0], _p(x), q.shape[0], _p(q), _p(p), float(sigma), _p(v))
    return v


def flow_points(q0, p0, x0, T, sigma):
    """Points x0 (M, 3) carried by the T Euler steps of the flow through the
    Eq. 4 velocity field; returns x(1)."""
    q0 = _in(q0); n = q0.shape[0]; p0 = _in(p0, n); x0 = _in(x0)
    x1 = np.empty_like(x0)
    _load().orc_flow_points(n, int(T), float(sigma), _p(q0), _p(p0), x0.shape[0], _p(x0), _p(x1))
    return x1


def _lbfgs_out(status, f, iters, evals, x, trace=None):
    out = dict(status=int(status), f=float(f.value), iters=int(iters.value), evals=int(evals.value), x=x)
    if trace is not None:
        out["trace"] = trace[: out["iters"] + 1].copy()
    return out


def lbfgs_quadratic(A, b, x0, m=10, max_iter=200, grad_tol=1e-12):
    """L-BFGS on 1/2 x^T A x - b^T x (pin helper)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64).ravel()
    x = np.ascontiguousarray(x0, dtype=np.float64).ravel().copy()
    f = ctypes.c_double(0); it = ctypes.c_int(0); ev = ctypes.c_int(0)
    st = _load().orc_lbfgs_quadratic(x.size, _p(A), _p(b), _p(x), int(m), int(max_iter), float(grad_tol),
                                     ctypes.byref(f), ctypes.byref(it), ctypes.byref(ev))
    return _lbfgs_out(st, f, it, ev, x)


def lbfgs_rosenbrock(x0, m=10, max_iter=500, grad_tol=1e-10):
    """L-BFGS on the extended Rosenbrock function (pin helper)."""
    x = np.ascontiguousarray(x0, dtype=np.float64).ravel().copy()
    f = ctypes.c_double(0); it = ctypes.c_int(0); ev = ctypes.c_int(0)
    st = _load().orc_lbfgs_rosenbrock(x.size, _p(x), int(m), int(max_iter), float(grad_tol),
                                      ctypes.byref(f), ctypes.byref(it), ctypes.byref(ev))
    return _lbfgs_out(st, f, it, ev, x)


def lbfgs_callback(fg, x0, m=10, max_iter=100, grad_tol=1e-10):
    """The oracle's L-BFGS (the one `register` runs) on a Python objective:
    fg(x) -> (f, g) with x, g 1-D float64 arrays.  For pins that observe every
    evaluation the optimiser makes."""
    x = np.ascontiguousarray(x0, dtype=np.float64).ravel().copy()
    n = x.size

    def cb(_ctx, xp, gp):
        xv = np.ctypeslib.as_array(xp, shape=(n,)).copy()
        f, g = fg(xv)
        np.ctypeslib.as_array(gp, shape=(n,))[:] = np.asarray(g, dtype=np.float64)
        return float(f)

    cfn = _FG(cb)
    f = ctypes.c_double(0); it = ctypes.c_int(0); ev = ctypes.c_int(0)
    st = _load().orc_lbfgs(n, _p(x), cfn, None, int(m), int(max_iter), float(grad_tol), ctypes.byref(f),
                           ctypes.byref(it), ctypes.byref(ev), None)
    return _lbfgs_out(st, f, it, ev, x)


def register(q0, target, T, sigma, lam, p0=None, m=10, max_iter=50, grad_tol=1e-5):
    """Algorithm 1, outer optimisation: L-BFGS over p0 of the Eq. 3 loss.  Returns
    dict(status, f, iters, evals, x=p0 (N,3), trace=loss per iterate)."""
    q0 = _in(q0); n = q0.shape[0]; target = _in(target, n)
    x = np.zeros((n, 3)) if p0 is None else _in(p0, n).copy()
    trace = np.zeros(max_iter + 1)
    f = ctypes.c_double(0); it = ctypes.c_int(0); ev = ctypes.c_int(0)
    st = _load().orc_register(n, int(T), float(sigma), float(lam), int(m), int(max_iter), float(grad_tol),
                              _p(q0), _p(target), _p(x), ctypes.byref(f), ctypes.byref(it), ctypes.byref(ev),
                              _p(trace))
    return _lbfgs_out(st, f, it, ev, x, trace)


# ---------------------------------------------------------------- variants
INTEGRATORS = {"euler": 0, "rk4": 1}
KINETIC = {"start": 0, "end": 1}


def _variant(integrator, h_at):
    if integrator not in INTEGRATORS or h_at not in KINETIC:
        raise ValueError("integrator must be one of %r and h_at one of %r" % (list(INTEGRATORS), list(KINETIC)))
    return INTEGRATORS[integrator], KINETIC[h_at]


def _in_d(a, n=None, dim=None):
    """(N, dim) float64 array with dim 2 or 3 (the dimension of the landmarks)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] not in (2, 3) or (n is not None and a.shape[0] != n) or (
            dim is not None and a.shape[1] != dim):
        raise ValueError("expected an (N, 2) or (N, 3) array, got shape %r" % (a.shape,))
    return a


def step_forward_d(q, p, sigma):
    """StepForward in 2-D or 3-D (the dimension of q): (Hq, Hp)."""
    q = _in_d(q); n, d = q.shape; p = _in_d(p, n, d)
    Hq = np.empty_like(q); Hp = np.empty_like(q)
    _load().orc_step_forward_d(d, n, float(sigma), _p(q), _p(p), _p(Hq), _p(Hp))
    return Hq, Hp


def step_backward_d(q, p, alpha, beta, sigma):
    """StepBackward in 2-D or 3-D: (dalpha, dbeta)."""
    q = _in_d(q); n, d = q.shape
    p, alpha, beta = _in_d(p, n, d), _in_d(alpha, n, d), _in_d(beta, n, d)
    da = np.empty_like(q); db = np.empty_like(q)
    _load().orc_step_backward_d(d, n, float(sigma), _p(q), _p(p), _p(alpha), _p(beta), _p(da), _p(db))
    return da, db


def hamiltonian_d(q, p, sigma) -> float:
    q = _in_d(q); n, d = q.shape; p = _in_d(p, n, d)
    return float(_load().orc_hamiltonian_d(d, n, float(sigma), _p(q), _p(p)))


def shoot_forward_v(q0, p0, T, sigma, integrator="euler"):
    """Forward flow with the chosen integrator ("euler" or "rk4"): (q1, p1).
    Landmarks in 2-D or 3-D (the shape of q0)."""
    ig, _ = _variant(integrator, "start")
    q0 = _in_d(q0); n, d = q0.shape; p0 = _in_d(p0, n, d)
    q1 = np.empty_like(q0); p1 = np.empty_like(q0)
    _load().orc_shoot_forward_v(d, n, int(T), float(sigma), ig, _p(q0), _p(p0), _p(q1), _p(p1))
    return q1, p1


def loss_v(q0, p0, target, T, sigma, lam, integrator="euler", h_at="start") -> float:
    """Loss of a variant: kinetic term at t = 0 ("start") or t = 1 ("end")."""
    ig, he = _variant(integrator, h_at)
    q0 = _in_d(q0); n, d = q0.shape
    p0, target = _in_d(p0, n, d), _in_d(target, n, d)
    return float(_load().orc_loss_v(d, n, int(T), float(sigma), float(lam), ig, he, _p(q0), _p(p0), _p(target)))


def shoot_gradient_v(q0, p0, target, T, sigma, lam, integrator="euler", h_at="start"):
    """ComputeGradient of a variant: dict(loss, grad_p0, grad_q0, q1, p1, H)
    with H the kinetic term of the loss.  2-D or 3-D landmarks."""
    ig, he = _variant(integrator, h_at)
    q0 = _in_d(q0); n, d = q0.shape
    p0, target = _in_d(p0, n, d), _in_d(target, n, d)
    gp = np.empty_like(q0); gq = np.empty_like(q0)
    q1 = np.empty_like(q0); p1 = np.empty_like(q0)
    h = ctypes.c_double(0.0)
    L = _load().orc_shoot_gradient_v(d, n, int(T), float(sigma), float(lam), ig, he, _p(q0), _p(p0), _p(target),
                                     _p(gp), _p(gq), _p(q1), _p(p1), ctypes.byref(h))
    return dict(loss=float(L), grad_p0=gp, grad_q0=gq, q1=q1, p1=p1, H=float(h.value))


def register_v(q0, target, T, sigma, lam, integrator="euler", h_at="start", p0=None, m=10, max_iter=50,
               grad_tol=1e-5):
    """register with a variant of the discretisation (2-D or 3-D landmarks)."""
    ig, he = _variant(integrator, h_at)
    q0 = _in_d(q0); n, d = q0.shape; target = _in_d(target, n, d)
    x = np.zeros((n, d)) if p0 is None else _in_d(p0, n, d).copy()
    trace = np.zeros(max_iter + 1)
    f = ctypes.c_double(0); it = ctypes.c_int(0); ev = ctypes.c_int(0)
    st = _load().orc_register_v(d, n, int(T), float(sigma), float(lam), ig, he, int(m), int(max_iter),
                                float(grad_tol), _p(q0), _p(target), _p(x), ctypes.byref(f), ctypes.byref(it),
                                ctypes.byref(ev), _p(trace))
    return _lbfgs_out(st, f, it, ev, x, trace)
