"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point include/gshoot.h declares.  No compute call is made
(there is no GPU here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gshoot.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:gs_status|const char\s*\*|void|int32_t)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("step_forward", "step_backward", "shoot_forward", "shoot_gradient", "gs_last_error"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert sorted(declared_functions()) == sorted(gsh.EXPORTS)
    assert lib.gs_version() >= 100


def test_params_struct_layout_matches_header():
    import paper_1907_04839_gb300 as gsh
    # int64 N, int32 T, int32 ckpt, double sigma, double lambda, int32 m,
    # int32 max_iter, double grad_tol  ->  48 bytes with natural alignment
    assert ctypes.sizeof(gsh.GsParams) == 48
    assert gsh.GsParams.sigma.offset == 16 and gsh.GsParams.grad_tol.offset == 40


def test_library_is_built_for_sm103a():
    import paper_1907_04839_gb300 as gsh
    from paper_1907_04839_gb300 import _build
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.LIB)


def test_no_cuda_device_is_reported_as_error_not_crash():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    import paper_1907_04839_gb300 as gsh
    q = np.zeros((4, 3), np.float32)
    with pytest.raises(gsh.GShootError):
        gsh.step_forward(q, q, 0.1)
