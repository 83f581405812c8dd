"""GPU test of step_forward_noalloc, the StepForward entry point for callers
that cannot allocate device memory.

Such a caller is, for example, a host program whose device memory belongs to
another allocator under a fixed budget, or code that must not pay for a
cudaMalloc, which can synchronise the whole device.  The entry point keeps
its scratch in a static device array instead of the library's workspace.
This test calls it through the C ABI twice in a row, on two different
problems, and checks each result against the ordinary step_forward entry
point, and against the FP64 oracle on the same FP32 inputs, within the 1e-5
normwise tolerance the parity tests use.  The file name makes pytest collect
it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel(a, b):
    a = a.double().cpu().numpy().ravel()
    b = b.double().cpu().numpy().ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_step_forward_noalloc_matches_step_forward_twice():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    # The larger problem first, so the second call runs on scratch that still
    # holds the first call's data.
    for n, sigma, seed in ((8192, 0.05, 11), (3001, 0.1, 12)):
        rng = np.random.default_rng(seed)
        q = torch.tensor(rng.uniform(-0.5, 0.5, size=(n, 3)), dtype=torch.float32, device="cuda")
        p = torch.tensor(rng.normal(0.0, 0.1, size=(n, 3)), dtype=torch.float32, device="cuda")
        Hq = torch.empty_like(q)
        Hp = torch.empty_like(q)
        st = lib.step_forward_noalloc(n, sigma, ptr(q), ptr(p), ptr(Hq), ptr(Hp), stream)
        assert st == 0, lib.gs_last_error().decode()
        ref_Hq, ref_Hp = gsh.step_forward(q, p, sigma)
        torch.cuda.synchronize()
        assert rel(Hp, ref_Hp) < 1e-5
        assert rel(Hq, ref_Hq) < 1e-5
        # the FP64 oracle on the same FP32 inputs
        import oracle
        o_Hq, o_Hp = oracle.step_forward(q.double().cpu().numpy(), p.double().cpu().numpy(), sigma)
        assert rel(Hp, torch.from_numpy(o_Hp)) < 1e-5
        assert rel(Hq, torch.from_numpy(o_Hq)) < 1e-5


def test_step_forward_noalloc_rejects_oversize_and_host_arrays():
    import paper_1907_04839_gb300 as gsh
    lib = gsh.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    big = torch.zeros((8193, 3), dtype=torch.float32, device="cuda")
    out = torch.empty_like(big)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.step_forward_noalloc(8193, 0.1, ptr(big), ptr(big), ptr(out), ptr(out), stream) == -1
    assert b"8192" in lib.gs_last_error()
    h = np.zeros((16, 3), dtype=np.float32)
    hp = ctypes.c_void_p(h.ctypes.data)
    assert lib.step_forward_noalloc(16, 0.1, hp, hp, hp, hp, stream) == -1
