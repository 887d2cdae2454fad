"""Stated parity tolerances per compute mode and output component.

Error metric (cancellation-aware, normwise): for output (p, c, i)
    err = |gpu - oracle| / size,   size = sum_k |C_ik| * size(chi_ck(p))
where size(chi) is the oracle's sum of the absolute values of the terms that
make up that AO entry.  Components: 0 value, 1-3 gradient, 4 Laplacian.

FP64: 1e-12 on every component.  The reduced modes carry the bounds derived
from their arithmetic (unit roundoff u = 2^-24 for FP32, 2^-9 per bf16
rounding, 2^-11 for TF32), each with the margin explained beside it.
"""
# mode -> (value, gradient, laplacian)
TOL = {
    # FP64 path: the spec bar
    "fp64": (1e-12, 1e-12, 1e-12),
    # FP32 AOs: __expf error <= (2 + 1.16 |t|) ulp with t < T <= 36, a dozen
    # roundings in the assembly, then an FP32 sum over K AOs whose error grows
    # like sqrt(K) u in practice; bound ~3e-6 + ~1e-5 -> stated 3e-5
    "fp32": (3e-5, 3e-5, 3e-5),
    # split bf16: each product keeps hi*hi + hi*lo + lo*hi; the dropped lo*lo
    # and the residuals of both splits are <= 3 * 2^-18 = 1.1e-5 of |x y|,
    # on top of the FP32 AO error above -> stated 5e-5
    "bf16x3": (5e-5, 5e-5, 5e-5),
    # TF32 keeps 10 explicit mantissa bits: <= 2 * 2^-11 per product -> 1e-3,
    # stated 3e-3
    "tf32": (3e-3, 3e-3, 3e-3),
}


def component_errors(got, ref, size):
    """Max normwise error for value, gradient (3 comps) and Laplacian."""
    import numpy as np
    e = np.abs(got - ref) / (size + 1e-300)
    return (float(e[:, 0].max()), float(e[:, 1:4].max()), float(e[:, 4].max()))


def assert_within(mode, got, ref, size, what=""):
    errs = component_errors(got, ref, size)
    tol = TOL[mode]
    names = ("value", "gradient", "laplacian")
    for n, e, t in zip(names, errs, tol):
        assert e <= t, f"{what} {mode} {n}: normwise error {e:.3e} > {t:.1e}"
    return errs
