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
                             stream=None, schedule=7, lane_split=0)
    h = ctypes.c_void_p(0)
    assert lib.gs_server_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
    assert b"schedule" in lib.gs_last_error()
    # a lane threshold only with the two-lane schedule, and never negative
    for sched, split in ((1, 4096), (2, -1)):
        cfg.schedule, cfg.lane_split = sched, split
        assert lib.gs_server_create(ctypes.byref(cfg), ctypes.byref(h)) == -1
        assert b"lane_split" in lib.gs_last_error()
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


def _table_rows():
    path = os.path.join(ROOT, "paper_1907_04839_gb300", "csrc", "step_table.inc")
    text = open(path).read()
    sms = int(re.search(r"kStepTableSms = (\d+);", text).group(1))
    rows = {int(m.group(1).split(",")[0]): tuple(int(v) for v in m.group(1).split(","))
            for m in re.finditer(r"^\s*\{([0-9, ]+)\},\s*$", text, re.M)}
    return sms, rows


def _step_config(lib, kind, n, sms, variants=0):
    t, c = ctypes.c_int32(0), ctypes.c_int32(0)
    assert lib.gs_step_config(kind, n, sms, variants, ctypes.byref(t), ctypes.byref(c)) == 0, lib.gs_last_error()
    return t.value, c.value


def _size_rule(kind, npad, variants=False):
    """The size rule the table refines: forward 128-thread CTAs in clusters of
    16, reverse 64-thread CTAs in clusters of 8; half-size CTAs up to 2048
    landmarks (reverse clusters of 16 up to 1024); clusters a power of two
    that leaves every CTA at least 8 sources."""
    threads, cmax = (128, 16) if kind == 0 else (64, 8)
    if not variants and npad <= 2048:
        threads //= 2
        if kind == 1 and npad <= 1024:
            cmax = 16
    cl = min(cmax, max(1, npad // 8))
    c = 1
    while c * 2 <= cl:
        c *= 2
    return threads, c


def test_step_config_follows_the_table_on_its_device():
    """gs_step_config (host logic only when the SM count is given) returns the
    table's row for every padded size the table covers (each N maps to the
    row of its padded count), the full-size CTAs' cluster for the variant
    kernels, and the size rule above the table."""
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    sms, rows = _table_rows()
    for n in list(range(1, 16385, 37)) + [64, 65, 2048, 4096, 16383, 16384]:
        npad = (n + 63) // 64 * 64
        r = rows[npad]
        assert _step_config(lib, 0, n, sms) == (r[1], r[2]), n
        assert _step_config(lib, 1, n, sms) == (r[4], r[5]), n
        assert _step_config(lib, 0, n, sms, 1) == (128, r[3]), n
        assert _step_config(lib, 1, n, sms, 1) == (64, r[6]), n
    for n in (16385, 20000, 65536, 1 << 20):
        npad = (n + 63) // 64 * 64
        for kind in (0, 1):
            assert _step_config(lib, kind, n, sms) == _size_rule(kind, npad), (kind, n)
            assert _step_config(lib, kind, n, sms, 1) == _size_rule(kind, npad, True), (kind, n)


def test_step_config_size_rule_without_the_table():
    """Another SM count, or the table switched off, gives the size rule."""
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    sms, _ = _table_rows()
    try:
        for other, on in ((sms - 20, 1), (sms, 0)):
            assert lib.gs_set_step_table(on) == 0
            for n in (1, 100, 1000, 1024, 1025, 2048, 2049, 3000, 4096, 7168, 16384, 70000):
                npad = (n + 63) // 64 * 64
                for kind in (0, 1):
                    assert _step_config(lib, kind, n, other) == _size_rule(kind, npad), (other, on, kind, n)
                    assert _step_config(lib, kind, n, other, 1) == _size_rule(kind, npad, True)
    finally:
        assert lib.gs_set_step_table(1) == 0


def test_step_config_override_applies_to_plain_launches_only():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    sms, rows = _table_rows()
    try:
        # reverse clusters that do not divide the tile exist for 32 / 64-thread CTAs only
        assert lib.gs_set_step_config(1, 128, 1, 1, 12) == -1
        assert lib.gs_set_step_config(1, 64, 1, 1, 12) == 0
        assert _step_config(lib, 1, 4096, sms) == (64, 12)
        assert _step_config(lib, 1, 40, sms) == (64, 8)  # at most npad / 8 CTAs per cluster
        assert _step_config(lib, 1, 4096, sms, 1) == (64, rows[4096][6])  # variants keep their kernels
        assert _step_config(lib, 0, 4096, sms) == (rows[4096][1], rows[4096][2])
    finally:
        assert lib.gs_set_step_config(1, 0, 0, 0, 0) == 0
    assert _step_config(lib, 1, 4096, sms) == (rows[4096][4], rows[4096][5])


def test_step_config_rejects_bad_arguments():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    t, c = ctypes.c_int32(0), ctypes.c_int32(0)
    assert lib.gs_step_config(2, 100, 152, 0, ctypes.byref(t), ctypes.byref(c)) == -1
    assert lib.gs_step_config(0, 0, 152, 0, ctypes.byref(t), ctypes.byref(c)) == -1
    assert lib.gs_step_config(0, (1 << 26) + 1, 152, 0, ctypes.byref(t), ctypes.byref(c)) == -1
    assert lib.gs_step_config(0, 100, 152, 0, None, ctypes.byref(c)) == -1


@pytest.mark.parametrize("mtype,ptr_dev,cur,want", [
    (0, -2, 0, 0),   # unregistered host memory: staged
    (1, 0, 0, 0),    # pinned host memory: staged
    (2, 0, 0, 1),    # device memory of the current GPU: used in place
    (2, 3, 3, 1),
    (2, 1, 0, 2),    # device memory of another GPU: rejected
    (2, 0, 5, 2),
    (3, 1, 0, 1),    # managed memory: used in place on any GPU
])
def test_pointer_rule_rejects_another_gpus_memory(mtype, ptr_dev, cur, want):
    # The rule every entry point applies to a caller's array, checked
    # without a GPU: memory of another device than the current one must be
    # refused, not handed to this device's kernels.
    import paper_1907_04839_gb300 as gsh
    assert gsh.load().gs_pointer_rule(mtype, ptr_dev, cur) == want


def test_batch_config_accepts_packed_shapes_only():
    # Host logic only: the packed kernels exist for one-group shapes whose
    # cluster divides the CTA; 0 restores the built-in shape.
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    try:
        assert lib.gs_set_batch_config(0, 128, 4) == 0
        assert lib.gs_set_batch_config(1, 64, 16) == 0
        assert lib.gs_set_batch_config(1, 32, 8) == 0
        assert lib.gs_set_batch_config(1, 64, 12) == -1   # does not divide the tile
        assert lib.gs_set_batch_config(0, 96, 8) == -1    # no such CTA size
        assert lib.gs_set_batch_config(0, 128, 32) == -1  # clusters of at most 16
        assert lib.gs_set_batch_config(2, 128, 8) == -1   # kind 0 or 1
    finally:
        assert lib.gs_set_batch_config(0, 0, 0) == 0
        assert lib.gs_set_batch_config(1, 0, 0) == 0


def test_combine_precision_switch_validates_its_argument():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    try:
        assert lib.gs_set_combine_precision(1) == 0
        assert lib.gs_set_combine_precision(2) == -1
        assert lib.gs_set_combine_precision(-1) == -1
    finally:
        assert lib.gs_set_combine_precision(0) == 0


def test_pair_loop_probe_rejects_bad_arguments():
    import ctypes
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    c = ctypes.c_double(0)
    for args in ((2, 64, 1, 1), (1, 48, 1, 1), (1, 288, 1, 1), (1, 256, 8, 1), (1, 64, 0, 1), (1, 64, 1, 0),
                 (1, 64, 1, 5000)):
        assert lib.gs_measure_pair_loop(*args, ctypes.byref(c), None) == -1, args
    assert lib.gs_measure_pair_loop(1, 64, 1, 1, None, None) == -1


def test_distinct_operand_probe_rejects_bad_arguments():
    import ctypes
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    d = ctypes.c_double(0)
    assert lib.gs_measure_ffma2_distinct(None, 20.0, None) == -1
    assert lib.gs_measure_ffma2_distinct(ctypes.byref(d), 0.5, None) == -1
    assert lib.gs_measure_ffma2_distinct(ctypes.byref(d), 5000.0, None) == -1
