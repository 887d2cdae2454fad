"""GB300-native AO/MO vgl evaluation (QMCkl method, arXiv 2512.16677).

The compute path is the CUDA library ``libqmckl_gpu.so`` (sources in
``csrc/``, ABI in ``include/qmckl_gpu.h``); ``qmckl`` is its ctypes binding
and ``autograd`` wraps the adjoint for PyTorch.  ``synth`` draws seeded
synthetic workloads.  Importing the package does not load the library;
the first ``qmckl.Context`` does, and raises if it has not been built.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "qmckl", "build"]


def build(force: bool = False) -> str:
    """Compile the CUDA library for sm_103a (in-tree)."""
    from .buildlib import build as _b
    return _b(force=force)
