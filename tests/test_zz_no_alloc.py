"""qk_contract_device_noalloc: the tensor-core contraction for callers that
cannot call cudaMalloc (a framework or pool owns the device memory, a
latency-critical loop cannot take the synchronisation of cudaMalloc/
cudaFree, or the caller must not fail for lack of memory once started).

Its result must match the FP64 product of its inputs, and the allocating
entry point qk_contract_device, within the contraction tolerances used
elsewhere in the tests, on two calls in a row (the shared scratch array
keeps the previous call's contents).  This
file is collected last so that a failure here comes after every other test.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"bf16x3": 3e-5, "tf32": 3e-3}     # same as tests/test_gpu_contract.py
MODES = {"bf16x3": 2, "tf32": 3}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_16677_gb300 import buildlib, qmckl
    buildlib.build()
    return qmckl.load()


def _call(lib, fn, mode, a, b, out):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return getattr(lib, fn)(MODES[mode], a.shape[0], b.shape[0], a.shape[1],
                            ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), stream)


def _inputs(seed, M, N, K):
    g = torch.Generator().manual_seed(seed)
    a = torch.randn(M, K, generator=g, dtype=torch.float32).cuda()
    b = torch.randn(N, K, generator=g, dtype=torch.float32).cuda()
    return a, b


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_noalloc_matches_allocating_entry(lib, mode):
    # two calls in a row with different shapes and data: the second must not
    # see anything of the first.  Each result is held against the FP64
    # product of its own inputs (normwise, the bar of the contraction tests)
    # and against the allocating entry point on the same inputs.
    for seed, (M, N, K) in ((1, (700, 300, 1650)), (2, (333, 37, 70))):
        a, b = _inputs(seed, M, N, K)
        ref = torch.empty(M, N, dtype=torch.float32, device="cuda")
        assert _call(lib, "qk_contract_device", mode, a, b, ref) == 0
        out = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
        assert _call(lib, "qk_contract_device_noalloc", mode, a, b, out) == 0
        torch.cuda.synchronize()
        a64, b64 = a.double().cpu(), b.double().cpu()
        exact = a64 @ b64.T
        size = a64.abs() @ b64.abs().T
        got = out.double().cpu()
        err64 = float(((got - exact).abs() / size).max())
        assert err64 <= TOL[mode], f"{mode} {(M, N, K)} vs FP64: {err64:.3e}"
        err = float(((got - ref.double().cpu()).abs() / size).max())
        assert err <= TOL[mode], f"{mode} {(M, N, K)} vs qk_contract_device: {err:.3e}"


def test_noalloc_rejects_oversize_and_bad_mode(lib):
    a, b = _inputs(3, 16, 16, 8)
    out = torch.zeros(16, 16, dtype=torch.float32, device="cuda")
    big_m = 3_000_000                      # (M + N) * ld far beyond the 32 MiB scratch
    st = lib.qk_contract_device_noalloc(2, big_m, 16, 8, ctypes.c_void_p(a.data_ptr()),
                                        ctypes.c_void_p(b.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), None)
    assert st == -3
    assert lib.qk_contract_device_noalloc(1, 16, 16, 8, ctypes.c_void_p(a.data_ptr()),
                                          ctypes.c_void_p(b.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), None) == -1
    assert torch.count_nonzero(out) == 0
