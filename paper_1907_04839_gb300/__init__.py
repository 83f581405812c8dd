"""gshoot: landmark matching by geodesic shooting on one GB300 (sm_103a).

A thin Python binding over the C ABI of ``libgshoot.so`` (include/gshoot.h).
The names are the same as in the ABI.  The binding only marshals arguments;
the CUDA kernels of the library do every step of the computation.

Arrays are (N, 3); shoot_forward, shoot_gradient, shoot and register also
take planar landmarks as (N, 2).  Two forms are accepted:
* torch CUDA tensors.  They are cast to contiguous float32, and the work runs
  on the current torch stream.  The outputs are CUDA tensors.
* numpy arrays or CPU tensors.  The library stages them through its device
  workspace and returns numpy float32 arrays.
"""
from __future__ import annotations

import contextlib
import ctypes

import numpy as np

from ._lib import (EXPORTS, INTEGRATORS, KINETIC_AT, GShootError, GsBatchProblem, GsParams, GsRegisterInfo,
                   GsServerConfig, check, load)

__all__ = [
    "step_forward", "step_backward", "shoot_forward", "shoot_gradient", "register", "shoot",
    "register_batch", "Server", "velocity_field", "flow_points",
    "release_workspace", "version", "GShootError", "GsParams", "EXPORTS",
]


def _is_cuda_tensor(x) -> bool:
    try:
        import torch
    except ImportError:  # pragma: no cover
        return False
    return isinstance(x, torch.Tensor) and x.is_cuda


def _dim_of(x) -> int:
    """2 for (N, 2) landmark arrays, else 3 (shapes are checked on marshalling)."""
    shape = tuple(x.shape)
    return 2 if len(shape) == 2 and shape[1] == 2 else 3


class _Marshal:
    """Pointers for one call: either all-device (torch) or all-host (numpy).
    Landmark arrays are (rows, dim) with dim 3, or 2 for planar landmarks."""

    def __init__(self, first, n=None, dim=3):
        self.device = _is_cuda_tensor(first)
        self.keep = []
        if self.device:
            import torch
            self.torch = torch
            self.dev = first.device
            self.stream = ctypes.c_void_p(torch.cuda.current_stream(self.dev).cuda_stream)
        else:
            self.stream = ctypes.c_void_p(0)
        self.n = n
        self.dim = dim

    def guard(self):
        """The device of the call's tensors made current while the library
        runs: the library uses the current device's workspace and rejects
        another GPU's memory."""
        if self.device:
            return self.torch.cuda.device(self.dev)
        return contextlib.nullcontext()

    def inp(self, x, name, rows=None):
        """Pointer to x as (rows, dim) FP32; rows defaults to the call's N."""
        if x is None:
            return None
        if self.device:
            if not _is_cuda_tensor(x):
                raise TypeError("%s: expected a CUDA tensor like the other inputs" % name)
            t = x.detach().to(device=self.dev, dtype=self.torch.float32).contiguous()
            arr_shape = tuple(t.shape)
            ptr = t.data_ptr()
        else:
            if hasattr(x, "detach"):
                x = x.detach().cpu().numpy()
            t = np.ascontiguousarray(x, dtype=np.float32)
            arr_shape = t.shape
            ptr = t.ctypes.data
        if len(arr_shape) != 2 or arr_shape[1] != self.dim:
            raise ValueError("%s: expected shape (N, %d), got %r" % (name, self.dim, arr_shape))
        if rows is not None:
            if arr_shape[0] != rows:
                raise ValueError("%s: expected %d rows, got %d" % (name, rows, arr_shape[0]))
        elif self.n is None:
            self.n = arr_shape[0]
        elif arr_shape[0] != self.n:
            raise ValueError("%s: expected %d rows, got %d" % (name, self.n, arr_shape[0]))
        self.keep.append(t)
        return ctypes.c_void_p(ptr)

    def out(self, rows=None):
        rows = self.n if rows is None else rows
        if self.device:
            t = self.torch.empty((rows, self.dim), dtype=self.torch.float32, device=self.dev)
            ptr = t.data_ptr()
        else:
            t = np.empty((rows, self.dim), dtype=np.float32)
            ptr = t.ctypes.data
        self.keep.append(t)
        return t, ctypes.c_void_p(ptr)


def _params(n, T, sigma, lam=0.0, ckpt_every=0, lbfgs_m=10, max_iter=100, grad_tol=1e-5, integrator="euler",
            h_at="start", dim=3):
    if integrator not in INTEGRATORS:
        raise ValueError("integrator must be one of %r" % sorted(INTEGRATORS))
    if h_at not in KINETIC_AT:
        raise ValueError("h_at must be one of %r" % sorted(KINETIC_AT))
    return GsParams(N=int(n), T=int(T), ckpt_every=int(ckpt_every), sigma=float(sigma),
                    lambda_=float(lam), lbfgs_m=int(lbfgs_m), max_iter=int(max_iter),
                    grad_tol=float(grad_tol), integrator=INTEGRATORS[integrator], kinetic_at=KINETIC_AT[h_at],
                    dim=int(dim), reserved=0)


def step_forward(q, p, sigma):
    """StepForward: returns (Hq, Hp), the two derivative terms of Eq. 2."""
    m = _Marshal(q)
    pq, pp = m.inp(q, "q"), m.inp(p, "p")
    Hq, oq = m.out()
    Hp, op = m.out()
    with m.guard():
        check(load().step_forward(m.n, float(sigma), pq, pp, oq, op, m.stream))
    return Hq, Hp


def velocity_field(q, p, x, sigma):
    """Eq. 4: the velocity of the landmark state (q, p) at points x (M, 3)."""
    m = _Marshal(q)
    pq, pp = m.inp(q, "q"), m.inp(p, "p")
    rows = int(x.shape[0])
    px = m.inp(x, "x", rows=rows)
    v, pv = m.out(rows=rows)
    with m.guard():
        check(load().velocity_field(m.n, rows, float(sigma), pq, pp, px, pv, m.stream))
    return v


def flow_points(q0, p0, x0, T, sigma):
    """Points x0 (M, 3) carried through the deformation that p0 generates:
    the same T Euler steps as the landmarks, through the Eq. 4 velocity
    field of each step.  Returns x(1)."""
    m = _Marshal(q0)
    pq, pp = m.inp(q0, "q0"), m.inp(p0, "p0")
    rows = int(x0.shape[0])
    px = m.inp(x0, "x0", rows=rows)
    x1, p1 = m.out(rows=rows)
    prm = _params(m.n, T, sigma)
    with m.guard():
        check(load().flow_points(ctypes.byref(prm), pq, pp, rows, px, p1, m.stream))
    return x1


def step_backward(q, p, alpha, beta, sigma):
    """StepBackward: returns (dalpha, dbeta), the adjoint pair sums of one
    reverse Euler step (alpha <- alpha + dt dalpha, beta <- beta + dt dbeta)."""
    m = _Marshal(q)
    pq, pp, pa, pb = m.inp(q, "q"), m.inp(p, "p"), m.inp(alpha, "alpha"), m.inp(beta, "beta")
    da, oa = m.out()
    db, ob = m.out()
    with m.guard():
        check(load().step_backward(m.n, float(sigma), pq, pp, pa, pb, oa, ob, m.stream))
    return da, db


def shoot_forward(q0, p0, T, sigma, integrator="euler"):
    """Forward flow of Algorithm 1: returns (q1, p1, H0) with H0 = H(p0, q0).
    integrator: "euler" (the paper's) or "rk4".  (N, 2) arrays: planar landmarks."""
    m = _Marshal(q0, dim=_dim_of(q0))
    pq, pp = m.inp(q0, "q0"), m.inp(p0, "p0")
    prm = _params(m.n, T, sigma, integrator=integrator, dim=m.dim)
    q1, o1 = m.out()
    p1, o2 = m.out()
    h0 = ctypes.c_double(0.0)
    with m.guard():
        check(load().shoot_forward(ctypes.byref(prm), pq, pp, o1, o2, ctypes.byref(h0), m.stream))
    return q1, p1, h0.value


def shoot_gradient(q0, p0, target, T, sigma, lam, ckpt_every=0, integrator="euler", h_at="start"):
    """ComputeGradient of Algorithm 1: returns (loss, dL/dp0, dL/dq0) for
    L = H(p0, q0) + lam ||q(1) - target||^2 (h_at="end": H(p(1), q(1))
    instead), with the flow integrated by "euler" or "rk4" steps.  (N, 2)
    arrays: planar landmarks."""
    m = _Marshal(q0, dim=_dim_of(q0))
    pq, pp, pt = m.inp(q0, "q0"), m.inp(p0, "p0"), m.inp(target, "target")
    prm = _params(m.n, T, sigma, lam, ckpt_every, integrator=integrator, h_at=h_at, dim=m.dim)
    gp, og = m.out()
    gq, oq = m.out()
    loss = ctypes.c_double(0.0)
    with m.guard():
        check(load().shoot_gradient(ctypes.byref(prm), pq, pp, pt, ctypes.byref(loss), og, oq, m.stream))
    return loss.value, gp, gq


_SHOOT_FN = None


def _shoot_function():
    """torch.autograd.Function over shoot_gradient (built on first use, so
    that the package imports without torch)."""
    global _SHOOT_FN
    if _SHOOT_FN is None:
        import torch

        class ShootLoss(torch.autograd.Function):
            @staticmethod
            def forward(ctx, q0, p0, target, T, sigma, lam, ckpt_every, integrator, h_at):
                loss, gp, gq = shoot_gradient(q0, p0, target, T, sigma, lam, ckpt_every, integrator, h_at)
                if not isinstance(gp, torch.Tensor):
                    gp, gq = torch.from_numpy(gp), torch.from_numpy(gq)
                ctx.save_for_backward(gq, gp)
                ctx.dtypes = (q0.dtype, p0.dtype)
                return torch.tensor(loss, dtype=torch.float64, device=q0.device)

            @staticmethod
            def backward(ctx, gout):
                gq, gp = ctx.saved_tensors
                dq = (gout.to(gq.dtype) * gq).to(ctx.dtypes[0]) if ctx.needs_input_grad[0] else None
                dp = (gout.to(gp.dtype) * gp).to(ctx.dtypes[1]) if ctx.needs_input_grad[1] else None
                return dq, dp, None, None, None, None, None, None, None

        _SHOOT_FN = ShootLoss
    return _SHOOT_FN


def shoot(q0, p0, target, T, sigma, lam, ckpt_every=0, integrator="euler", h_at="start"):
    """The loss of Eq. 3 as a differentiable torch scalar (FP64).

    Backward gives dL/dq0 and dL/dp0 (no gradient flows to ``target``).  Both
    come from the same library call as the loss: the forward flow, the loss,
    and the exact reverse sweep of the time steps ("euler" or "rk4"; h_at
    places the kinetic term at t = 0 or t = 1).  With ``ckpt_every = k``
    (0 < k < T), the reverse sweep keeps the state only every k steps and
    recomputes the rest.  The results are bitwise identical."""
    return _shoot_function().apply(q0, p0, target, T, sigma, lam, ckpt_every, integrator, h_at)


def register(q0, target, T, sigma, lam, p0=None, m=10, max_iter=100, grad_tol=1e-5, integrator="euler",
             h_at="start"):
    """Algorithm 1, outer optimisation: L-BFGS over p0 of the Eq. 3 loss.  Returns
    (p0, info) with info a dict (loss, grad_norm0, grad_norm, avg_dist,
    max_dist, iters, evals, status).  integrator / h_at select the variant
    of the discretisation as in shoot_gradient.  (N, 2) arrays: planar landmarks."""
    m_ = _Marshal(q0, dim=_dim_of(q0))
    pq, pt = m_.inp(q0, "q0"), m_.inp(target, "target")
    if p0 is None:
        p0 = np.zeros((m_.n, m_.dim), np.float32) if not m_.device else m_.torch.zeros(
            (m_.n, m_.dim), dtype=m_.torch.float32, device=m_.dev)
    if m_.device:
        pout = p0.detach().to(device=m_.dev, dtype=m_.torch.float32).clone().contiguous()
        pp = ctypes.c_void_p(pout.data_ptr())
    else:
        pout = np.array(p0.detach().cpu().numpy() if hasattr(p0, "detach") else p0, dtype=np.float32, copy=True)
        pp = ctypes.c_void_p(pout.ctypes.data)
    if tuple(pout.shape) != (m_.n, m_.dim):
        raise ValueError("p0: expected shape (%d, %d)" % (m_.n, m_.dim))
    prm = _params(m_.n, T, sigma, lam, 0, m, max_iter, grad_tol, integrator, h_at, m_.dim)
    info = GsRegisterInfo()
    with m_.guard():
        check(load().register_landmarks(ctypes.byref(prm), pq, pt, pp, ctypes.byref(info), m_.stream))
    return pout, info.as_dict()


def _host_f32(x, n=None):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    a = np.ascontiguousarray(x, dtype=np.float32)
    if a.ndim != 2 or a.shape[1] != 3 or (n is not None and a.shape[0] != n):
        raise ValueError("expected an (N, 3) array")
    return a


def register_batch(problems, T, m=10, max_iter=100, grad_tol=1e-5, stream=None):
    """Run register over many independent problems at once (packed launches).

    ``problems`` is a list of dicts with keys q0, target, sigma, lam and
    optionally p0 (host arrays or tensors).  Returns a list of (p0, info)."""
    keep = []
    arr = (GsBatchProblem * len(problems))()
    outs = []
    for k, pr in enumerate(problems):
        q0 = _host_f32(pr["q0"])
        n = q0.shape[0]
        t = _host_f32(pr["target"], n)
        p0 = _host_f32(pr["p0"], n).copy() if pr.get("p0") is not None else np.zeros((n, 3), np.float32)
        keep += [q0, t, p0]
        outs.append(p0)
        arr[k].N = n
        arr[k].sigma = float(pr["sigma"])
        arr[k].lambda_ = float(pr["lam"])
        arr[k].q0 = q0.ctypes.data
        arr[k].target = t.ctypes.data
        arr[k].p0 = p0.ctypes.data
    check(load().register_batch(len(problems), arr, int(T), int(m), int(max_iter), float(grad_tol),
                                ctypes.c_void_p(stream or 0)))
    return [(outs[k], arr[k].info.as_dict()) for k in range(len(problems))]


class Server:
    """Continuous-batching registration server (gs_server_* in the C ABI).

    submit() queues a request; step() runs one round (admission by memory
    budget, one evaluation of each request the schedule selects, retirement);
    poll() returns (p0, info, latency) of a finished request or None.
    schedule "fair" (the default) shares pair work equally among resident
    requests, so small ones finish sooner; "all" evaluates every resident
    request in every round; "lanes" runs requests of at most `lane_split`
    landmarks (0: 8192) in a second, fair-scheduled engine concurrently with
    the all-rounds engine of the larger ones."""

    def __init__(self, T, m=10, max_iter=100, grad_tol=1e-5, memory_budget=8 << 30, max_problems=1024,
                 stream=None, schedule="fair", lane_split=0):
        schedules = {"all": 0, "fair": 1, "lanes": 2}
        if schedule not in schedules:
            raise ValueError("schedule must be 'all', 'fair' or 'lanes'")
        self._lib = load()
        cfg = GsServerConfig(T=int(T), lbfgs_m=int(m), max_iter=int(max_iter), max_problems=int(max_problems),
                             grad_tol=float(grad_tol), memory_budget=int(memory_budget),
                             stream=ctypes.c_void_p(stream or 0), schedule=schedules[schedule],
                             lane_split=int(lane_split))
        self._h = ctypes.c_void_p(0)
        check(self._lib.gs_server_create(ctypes.byref(cfg), ctypes.byref(self._h)))
        self._n = {}

    def submit(self, q0, target, sigma, lam, p0=None):
        q0 = _host_f32(q0)
        n = q0.shape[0]
        t = _host_f32(target, n)
        p = _host_f32(p0, n) if p0 is not None else None
        rid = ctypes.c_int64(0)
        check(self._lib.gs_server_submit(self._h, n, float(sigma), float(lam), q0.ctypes.data, t.ctypes.data,
                                         p.ctypes.data if p is not None else None, ctypes.byref(rid)))
        self._n[rid.value] = n
        return rid.value

    def step(self):
        a, q, c = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_int32(0)
        check(self._lib.gs_server_step(self._h, ctypes.byref(a), ctypes.byref(q), ctypes.byref(c)))
        return a.value, q.value, c.value

    def poll(self, rid):
        n = self._n[rid]
        p0 = np.empty((n, 3), np.float32)
        info = GsRegisterInfo()
        lat = (ctypes.c_double * 2)()
        done = ctypes.c_int32(0)
        check(self._lib.gs_server_poll(self._h, int(rid), p0.ctypes.data, ctypes.byref(info), lat,
                                       ctypes.byref(done)))
        if not done.value:
            return None
        return p0, info.as_dict(), (lat[0], lat[1])

    def stats(self):
        c, f, b = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
        check(self._lib.gs_server_stats(self._h, ctypes.byref(c), ctypes.byref(f), ctypes.byref(b)))
        return {"capacity_landmarks": c.value, "free_landmarks": f.value, "bytes": b.value}

    def close(self):
        if self._h:
            self._lib.gs_server_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def release_workspace() -> None:
    load().gs_release_workspace()


def version() -> int:
    return int(load().gs_version())
