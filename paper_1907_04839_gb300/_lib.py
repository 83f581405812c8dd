"""ctypes loader for libgshoot.so (the C ABI declared in include/gshoot.h).

There is no fallback.  If the library cannot be built or loaded, every entry
point raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

_lock = threading.Lock()
_lib = None

GS_STATUS = {
    0: "GS_OK", 1: "GS_NOT_CONVERGED", -1: "GS_EINVAL", -2: "GS_ENOMEM", -3: "GS_ECUDA",
    -4: "GS_ETIMEOUT", -5: "GS_ENONFINITE", -6: "GS_ENOLIB",
}

# Every symbol the header declares; tests check the library exports them all.
EXPORTS = [
    "step_forward", "step_backward", "shoot_forward", "shoot_gradient", "register_landmarks",
    "velocity_field", "flow_points",
    "register_batch", "gs_server_create", "gs_server_submit", "gs_server_step", "gs_server_poll",
    "gs_server_stats", "gs_server_destroy",
    "gs_time_pair_kernels", "gs_time_pair_config", "gs_set_step_config", "step_forward_noalloc",
    "gs_set_phase_timing", "gs_phase_times", "gs_set_cluster_policy", "gs_max_active_clusters",
    "gs_set_late_trigger", "gs_check_wait_timeout", "gs_set_step_table", "gs_step_config",
    "gs_pointer_rule", "gs_measure_peaks", "gs_set_combine_precision",
    "gs_set_batch_config", "gs_measure_pair_loop", "gs_measure_ffma2_distinct",
    "gs_last_error",
    "gs_release_workspace",
    "gs_version",
]


class GsParams(ctypes.Structure):
    """Mirror of ``gs_params`` in include/gshoot.h."""
    _fields_ = [
        ("N", ctypes.c_int64),
        ("T", ctypes.c_int32),
        ("ckpt_every", ctypes.c_int32),
        ("sigma", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("lbfgs_m", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("grad_tol", ctypes.c_double),
        ("integrator", ctypes.c_int32),
        ("kinetic_at", ctypes.c_int32),
        ("dim", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]


# gs_params.integrator and gs_params.kinetic_at values (include/gshoot.h).
INTEGRATORS = {"euler": 0, "rk4": 1}
KINETIC_AT = {"start": 0, "end": 1}


class GsRegisterInfo(ctypes.Structure):
    """Mirror of ``gs_register_info`` in include/gshoot.h."""
    _fields_ = [
        ("loss", ctypes.c_double),
        ("grad_norm0", ctypes.c_double),
        ("grad_norm", ctypes.c_double),
        ("avg_dist", ctypes.c_double),
        ("max_dist", ctypes.c_double),
        ("iters", ctypes.c_int32),
        ("evals", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class GsBatchProblem(ctypes.Structure):
    """Mirror of ``gs_batch_problem``."""
    _fields_ = [
        ("N", ctypes.c_int64),
        ("sigma", ctypes.c_double),
        ("lambda_", ctypes.c_double),
        ("q0", ctypes.c_void_p),
        ("target", ctypes.c_void_p),
        ("p0", ctypes.c_void_p),
        ("info", GsRegisterInfo),
    ]


class GsServerConfig(ctypes.Structure):
    """Mirror of ``gs_server_config``."""
    _fields_ = [
        ("T", ctypes.c_int32),
        ("lbfgs_m", ctypes.c_int32),
        ("max_iter", ctypes.c_int32),
        ("max_problems", ctypes.c_int32),
        ("grad_tol", ctypes.c_double),
        ("memory_budget", ctypes.c_uint64),
        ("stream", ctypes.c_void_p),
        ("schedule", ctypes.c_int32),
        ("lane_split", ctypes.c_int32),
    ]


class GShootError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (GS_STATUS.get(status, "?"), status, msg))
        self.status = status


def _declare(lib):
    vp, fp, dp, i64, i32, cd = (ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_int64, ctypes.c_int32, ctypes.c_double)
    P = ctypes.POINTER(GsParams)
    lib.step_forward.argtypes = [i64, cd, fp, fp, fp, fp, vp]
    lib.step_backward.argtypes = [i64, cd, fp, fp, fp, fp, fp, fp, vp]
    lib.shoot_forward.argtypes = [P, fp, fp, fp, fp, dp, vp]
    lib.shoot_gradient.argtypes = [P, fp, fp, fp, dp, fp, fp, vp]
    lib.register_landmarks.argtypes = [P, fp, fp, fp, ctypes.POINTER(GsRegisterInfo), vp]
    lib.velocity_field.argtypes = [i64, i64, cd, fp, fp, fp, fp, vp]
    lib.flow_points.argtypes = [P, fp, fp, i64, fp, fp, vp]
    lib.register_batch.argtypes = [i32, ctypes.POINTER(GsBatchProblem), i32, i32, i32, cd, vp]
    lib.register_batch.restype = ctypes.c_int
    SV = ctypes.c_void_p
    lib.gs_server_create.argtypes = [ctypes.POINTER(GsServerConfig), ctypes.POINTER(SV)]
    lib.gs_server_submit.argtypes = [SV, i64, cd, cd, fp, fp, fp, ctypes.POINTER(ctypes.c_int64)]
    lib.gs_server_step.argtypes = [SV, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.gs_server_poll.argtypes = [SV, ctypes.c_int64, fp, ctypes.POINTER(GsRegisterInfo),
                                   ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
    lib.gs_server_stats.argtypes = [SV, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                    ctypes.POINTER(ctypes.c_int64)]
    lib.gs_server_destroy.argtypes = [SV]
    lib.gs_server_destroy.restype = None
    for name in ("gs_server_create", "gs_server_submit", "gs_server_step", "gs_server_poll", "gs_server_stats"):
        getattr(lib, name).restype = ctypes.c_int
    lib.gs_time_pair_kernels.argtypes = [P, fp, fp, fp, i32, dp, dp, ctypes.c_void_p, vp]
    lib.step_forward_noalloc.argtypes = [i64, cd, fp, fp, fp, fp, vp]
    lib.gs_set_step_config.argtypes = [i32, i32, i32, i32, i32]
    lib.gs_set_phase_timing.argtypes = [i32]
    lib.gs_set_cluster_policy.argtypes = [i32]
    lib.gs_set_late_trigger.argtypes = [i32]
    lib.gs_set_step_table.argtypes = [i32]
    lib.gs_step_config.argtypes = [i32, ctypes.c_int64, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.gs_check_wait_timeout.argtypes = [i32, dp, vp]
    lib.gs_max_active_clusters.argtypes = [i32, i32, i32, i32, i32, ctypes.c_void_p]
    lib.gs_phase_times.argtypes = [dp, dp]
    lib.gs_time_pair_config.argtypes = [i32, i64, cd, fp, fp, fp, fp, i32, i32, i32, i32, i32, dp,
                                        ctypes.c_void_p, vp]
    for name in ("step_forward", "step_backward", "shoot_forward", "shoot_gradient", "register_landmarks",
                 "velocity_field", "flow_points",
                 "gs_time_pair_kernels",
                 "step_forward_noalloc", "gs_time_pair_config", "gs_set_step_config", "gs_set_phase_timing",
                 "gs_phase_times", "gs_set_cluster_policy", "gs_max_active_clusters", "gs_set_late_trigger",
                 "gs_set_step_table", "gs_step_config", "gs_check_wait_timeout", "gs_measure_peaks",
                 "gs_set_combine_precision", "gs_set_batch_config", "gs_measure_pair_loop",
                 "gs_measure_ffma2_distinct"):
        getattr(lib, name).restype = ctypes.c_int
    lib.gs_last_error.restype = ctypes.c_char_p
    lib.gs_last_error.argtypes = []
    lib.gs_release_workspace.restype = None
    lib.gs_version.restype = i32
    lib.gs_measure_peaks.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                     ctypes.c_double, ctypes.c_void_p]
    lib.gs_pointer_rule.restype = i32
    lib.gs_pointer_rule.argtypes = [i32, i32, i32]
    lib.gs_measure_pair_loop.argtypes = [i32, i32, i32, i32, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    lib.gs_measure_ffma2_distinct.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.c_double, ctypes.c_void_p]


def load(build_if_missing: bool = True):
    """Load libgshoot.so, building it first if it is absent or stale."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError("libgshoot.so is not built; run paper_1907_04839_gb300._build.build()")
            lib = ctypes.CDLL(path)
            _declare(lib)
            _lib = lib
    return _lib


def check(status: int) -> int:
    if status < 0:
        raise GShootError(status, load().gs_last_error().decode(errors="replace"))
    return status
