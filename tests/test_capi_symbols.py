"""CPU checks of the boundary: the library builds for sm_103a, loads, and
exports every entry point include/gshoot.h declares.  No compute call is made
(there is no GPU here)."""
import ctypes
import os
import re
import subprocess

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


def test_params_struct_layout_matches_header(tmp_path):
    # The ctypes mirror against the C compiler's own layout of the header.
    import paper_1907_04839_gb300 as gsh
    fields = [f[0] for f in gsh.GsParams._fields_]
    cnames = {"lambda_": "lambda"}
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"gshoot.h\"\nint main(void) {\n"
                   + '  printf("%zu\\n", sizeof(gs_params));\n'
                   + "".join('  printf("%%zu\\n", offsetof(gs_params, %s));\n' % cnames.get(f, f) for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(gsh.GsParams)
    assert out[1:] == [getattr(gsh.GsParams, f).offset for f in fields]


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


def test_invalid_variant_is_rejected_before_device_work():
    import numpy as np
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    q = np.zeros((4, 3), np.float32)
    for integ, kin in ((2, 0), (0, 2), (-1, 0)):
        prm = gsh.GsParams(N=4, T=2, ckpt_every=0, sigma=0.1, lambda_=1.0, lbfgs_m=10, max_iter=1, grad_tol=0.0,
                           integrator=integ, kinetic_at=kin)
        P = lambda a: ctypes.c_void_p(a.ctypes.data)
        st = lib.shoot_gradient(ctypes.byref(prm), P(q), P(q), P(q), None, P(q), P(q), None)
        assert st == -1, (integ, kin, st)
        assert b"integrator" in lib.gs_last_error() or b"kinetic_at" in lib.gs_last_error()


def test_invalid_dimension_and_server_schedule_are_rejected():
    import numpy as np
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    q = np.zeros((4, 3), np.float32)
    P = lambda a: ctypes.c_void_p(a.ctypes.data)
    for dim in (1, 4, -3):
        prm = gsh.GsParams(N=4, T=2, ckpt_every=0, sigma=0.1, lambda_=1.0, lbfgs_m=10, max_iter=1, grad_tol=0.0,
                           integrator=0, kinetic_at=0, dim=dim, reserved=0)
        assert lib.shoot_forward(ctypes.byref(prm), P(q), P(q), P(q), P(q), None, None) == -1
        assert b"dim" in lib.gs_last_error()
    cfg = gsh.GsServerConfig(T=4, lbfgs_m=10, max_iter=1, max_problems=1, grad_tol=0.0, memory_budget=1 << 20,
                             stream=None, schedule=7, reserved=0)
    h = ctypes.c_void_p(0)
    assert lib.gs_server_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert b"schedule" in lib.gs_last_error()
    with pytest.raises(ValueError):
        gsh.Server(T=4, schedule="sometimes")


def test_server_config_layout_matches_header(tmp_path):
    import paper_1907_04839_gb300 as gsh
    fields = [f[0] for f in gsh.GsServerConfig._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stdio.h>\n#include <stddef.h>\n#include \"gshoot.h\"\nint main(void) {\n"
                   + '  printf("%zu\\n", sizeof(gs_server_config));\n'
                   + "".join('  printf("%%zu\\n", offsetof(gs_server_config, %s));\n' % f for f in fields)
                   + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(gsh.GsServerConfig)
    assert out[1:] == [getattr(gsh.GsServerConfig, f).offset for f in fields]


def test_step_table_switch_rejects_other_values():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    for bad in (-1, 2, 7):
        assert lib.gs_set_step_table(bad) == -1
        assert b"on must be" in lib.gs_last_error()


def test_step_table_rows_are_valid_configurations():
    """Every row of the compiled-in step-configuration table names a kernel
    that exists (forward 64 / 128 threads, reverse 32 / 64) and a cluster of
    at most 16 CTAs, no more than the CTA's targets, that leaves every CTA of
    the cluster at least 8 sources; the rows ascend."""
    import re
    path = os.path.join(ROOT, "paper_1907_04839_gb300", "csrc", "step_table.inc")
    text = open(path).read()
    sms = int(re.search(r"kStepTableSms = (\d+);", text).group(1))
    assert sms > 0
    rows = [tuple(int(v) for v in m.group(1).split(","))
            for m in re.finditer(r"^\s*\{([0-9, ]+)\},\s*$", text, re.M)]
    assert len(rows) >= 256
    npads = [r[0] for r in rows]
    assert npads == sorted(npads) and len(set(npads)) == len(npads)
    assert npads == list(range(64, 16384 + 1, 64))
    for npad, ft, fc, ffc, bt, bc, bfc in rows:
        assert ft in (64, 128) and bt in (32, 64)
        for threads, c in ((ft, fc), (128, ffc), (bt, bc), (64, bfc)):
            assert 1 <= c <= 16 and c <= threads and c <= max(1, npad // 8), (npad, threads, c)
