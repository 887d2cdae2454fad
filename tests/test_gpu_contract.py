"""Each contraction kernel alone (qk_contract_device): D = A B^T.

The reference is the plain definition, a float64 matrix product of the same
inputs.  Shapes are ragged against every tile (M vs 128 rows, N vs the MMA
width, K vs the 64-element K block), and a one-hot A checks the layout:
row m of D must be column k(m) of B.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# normwise bound |D - ref| / (|A| |B|^T) per mode (see tests/tolerances.py)
TOL = {"fp64": 1e-14, "fp32": 2e-5, "bf16x3": 3e-5, "tf32": 3e-3}
# MO counts on either side of the 160-column N tile and of two of them
SHAPES = [(128, 16, 64), (200, 37, 70), (1000, 5, 25), (257, 256, 129), (300, 100, 500),
          (513, 300, 1650), (390, 161, 200), (129, 304, 96), (200, 320, 300)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_16677_gb300 import buildlib
    buildlib.build()


def _run(A, B, mode):
    from paper_2512_16677_gb300 import qmckl
    dt = torch.float64 if mode == "fp64" else torch.float32
    a = torch.from_numpy(A).to(dt).cuda().contiguous()
    b = torch.from_numpy(B).to(dt).cuda().contiguous()
    d = qmckl.contract_device(a, b, mode)
    torch.cuda.synchronize()
    return d.double().cpu().numpy()


@pytest.mark.parametrize("mode", ["fp64", "fp32", "bf16x3", "tf32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_random(mode, shape):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.normal(size=(M, K)) * np.exp(rng.uniform(-3, 3, size=(M, 1)))
    B = rng.normal(size=(N, K))
    if mode != "fp64":     # the kernels read FP32 inputs
        A = A.astype(np.float32).astype(np.float64)
        B = B.astype(np.float32).astype(np.float64)
    got = _run(A, B, mode)
    ref = A @ B.T
    size = np.abs(A) @ np.abs(B).T
    err = float(np.max(np.abs(got - ref) / size))
    assert err <= TOL[mode], f"{mode} {shape}: {err:.3e}"


@pytest.mark.parametrize("mode", ["bf16x3", "tf32", "fp32"])
def test_one_hot_layout(mode):
    M, N, K = 390, 300, 1650
    rng = np.random.default_rng(11)
    ks = rng.integers(0, K, size=M)
    A = np.zeros((M, K))
    A[np.arange(M), ks] = 1.0
    B = rng.normal(size=(N, K)).astype(np.float32).astype(np.float64)
    got = _run(A, B, mode)
    ref = B[:, ks].T
    np.testing.assert_allclose(got, ref, rtol=TOL[mode], atol=TOL[mode] * np.abs(ref).max())
