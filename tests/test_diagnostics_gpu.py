"""GPU tests of the measurement diagnostics behind the roofline figures:
gs_measure_peaks (unit throughputs) and gs_measure_pair_loop (the pair
loops alone).  Their outputs must respect the bounds the hardware's unit
counts fix: no FP32 rate above 152 SMs x 128 lanes x 2 flops at the
maximum clock, and no loop faster than its paired FP32 instructions can
pass through the pipe (two cycles each)."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def lib_and_stream():
    import paper_1907_04839_gb300 as gsh
    return gsh.load(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_measured_peaks_respect_the_unit_counts():
    lib, st = lib_and_stream()
    props = torch.cuda.get_device_properties(0)
    rates = (ctypes.c_double * 4)()
    ms = (ctypes.c_double * 4)()
    assert lib.gs_measure_peaks(rates, ms, 20.0, st) == 0, lib.gs_last_error()
    bound = props.multi_processor_count * 128 * 2 * 2.2e9 * 1e-12  # TFLOP/s at a 2.2 GHz ceiling
    print(list(rates), list(ms))
    assert 0.25 * bound < rates[0] <= bound
    assert 0.25 * bound < rates[1] <= bound
    assert rates[2] > 1e11
    assert 0.0 < rates[3] < rates[1]


@pytest.mark.parametrize("kind,instr", [(0, 16), (1, 36)])
def test_pair_loop_probe_respects_the_pipe_bound(kind, instr):
    lib, st = lib_and_stream()
    out = {}
    for ctas in (2, 4, 8):  # 1, 2 and 4 warps per scheduler with 64-thread CTAs
        c = ctypes.c_double(0)
        assert lib.gs_measure_pair_loop(kind, 64, ctas, 16, ctypes.byref(c), st) == 0, lib.gs_last_error()
        out[ctas] = c.value
    print(kind, out)
    for ctas, cyc in out.items():
        wps = ctas * 64 / 128
        assert cyc >= 0.95 * 2 * instr * wps  # the pipe passes one paired instruction per two cycles
        assert cyc < 50 * 2 * instr * wps
    assert out[8] >= out[4] >= 0.9 * out[2]  # warps sharing a scheduler never speed one another up


def test_distinct_operand_ffma2_rate_is_below_the_shared_operand_rate():
    lib, st = lib_and_stream()
    rates = (ctypes.c_double * 4)()
    assert lib.gs_measure_peaks(rates, None, 20.0, st) == 0, lib.gs_last_error()
    d = ctypes.c_double(0)
    assert lib.gs_measure_ffma2_distinct(ctypes.byref(d), 20.0, st) == 0, lib.gs_last_error()
    print(rates[1], d.value)
    assert 0.25 * rates[1] < d.value <= 1.02 * rates[1]
