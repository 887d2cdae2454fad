"""ctypes front end of the FP64 CPU oracle in ``oracle.c``.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are its only callers.  It imports nothing
from the CUDA library's package: inputs arrive as ``synth.Molecule``-like
objects (plain numpy arrays) drawn by the seeded input generator.

Functions and the passage they follow:

* ``threshold``      Eq. 3: T = (B-1) ln 2, or ln(1/eps) for an explicit cutoff
* ``ao_vgl``         Eqs. 1, 2, 4 with gradients and Laplacians (Sec. 3.1)
* ``mo_vgl``         Eqs. 5-7 (Sec. 3.2), compensated (Dot2) sums
* ``mo_from_ao``     Eqs. 5-7 applied to a given AO tensor
* ``adjoint``        dL/dC and dL/dR_nuc of L = sum W * mo_vgl (Sec. 3.6 asks
                     for nuclear derivatives up to third order)
* ``screen_counts``  how many (point, shell) pairs and primitives pass Eq. 3
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import sys
from typing import Optional, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
LIB = os.path.join(HERE, "liboracle.so")

CFLAGS = ["-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
          "-fno-fast-math"]


def build(force: bool = False, src: str = SRC, out: str = LIB) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, portable flags)."""
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(src)):
        return out
    tmp = f"{out}.{os.getpid()}.tmp"
    subprocess.check_call(["gcc", *CFLAGS, src, "-o", tmp, "-lm"])
    os.replace(tmp, out)
    return out


class _Basis(ctypes.Structure):
    _fields_ = [
        ("nucl_num", ctypes.c_int64), ("nucl_coord", ctypes.c_void_p),
        ("shell_num", ctypes.c_int64), ("shell_nucleus", ctypes.c_void_p),
        ("shell_ang_mom", ctypes.c_void_p), ("shell_prim_num", ctypes.c_void_p),
        ("shell_factor", ctypes.c_void_p),
        ("prim_num", ctypes.c_int64), ("exponent", ctypes.c_void_p),
        ("coefficient", ctypes.c_void_p), ("prim_factor", ctypes.c_void_p),
        ("ao_num", ctypes.c_int64), ("ao_factor", ctypes.c_void_p),
    ]


_lib = None


def _load():
    global _lib
    if _lib is None:
        # ORACLE_LIB points at another build of oracle.c (the mutation tests
        # load deliberately broken copies through it)
        path = os.environ.get("ORACLE_LIB") or build()
        lib = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I = ctypes.c_int64
        D = ctypes.c_double
        lib.oracle_threshold_bits.restype = D
        lib.oracle_threshold_bits.argtypes = [ctypes.c_int]
        lib.oracle_threshold_eps.restype = D
        lib.oracle_threshold_eps.argtypes = [D]
        lib.oracle_ao_vgl.argtypes = [P, D, I, P, P, P]
        lib.oracle_mo_vgl.argtypes = [I, I, P, I, P, P, P, P]
        lib.oracle_mo_vgl_points.argtypes = [P, D, I, P, I, P, P, P]
        lib.oracle_adjoint.argtypes = [P, D, I, P, I, P, P, P, P, P, P]
        lib.oracle_screen_counts.argtypes = [P, D, I, P, P]
        for f in ("oracle_ao_vgl", "oracle_mo_vgl", "oracle_mo_vgl_points",
                  "oracle_adjoint", "oracle_screen_counts"):
            getattr(lib, f).restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class _BasisRef:
    """Keeps the numpy arrays behind a _Basis struct alive."""

    def __init__(self, mol, nucl_coord=None):
        self.arrs = dict(
            nucl_coord=_c(mol.nucl_coord if nucl_coord is None else nucl_coord, np.float64),
            shell_nucleus=_c(mol.shell_nucleus, np.int64),
            shell_ang_mom=_c(mol.shell_ang_mom, np.int32),
            shell_prim_num=_c(mol.shell_prim_num, np.int64),
            shell_factor=_c(mol.shell_factor, np.float64),
            exponent=_c(mol.exponent, np.float64),
            coefficient=_c(mol.coefficient, np.float64),
            prim_factor=_c(mol.prim_factor, np.float64),
            ao_factor=_c(mol.ao_factor, np.float64),
        )
        a = self.arrs
        self.ao_num = int(a["ao_factor"].shape[0])
        self.s = _Basis(
            a["nucl_coord"].shape[0], _ptr(a["nucl_coord"]),
            a["shell_ang_mom"].shape[0], _ptr(a["shell_nucleus"]),
            _ptr(a["shell_ang_mom"]), _ptr(a["shell_prim_num"]), _ptr(a["shell_factor"]),
            a["exponent"].shape[0], _ptr(a["exponent"]), _ptr(a["coefficient"]),
            _ptr(a["prim_factor"]), self.ao_num, _ptr(a["ao_factor"]))

    @property
    def ref(self):
        return ctypes.byref(self.s)


def threshold(mol, screened: bool = True) -> float:
    """Eq. 3 threshold on gamma * r^2 (math.inf when unscreened)."""
    if not screened:
        return math.inf
    lib = _load()
    if getattr(mol, "eps", None) is not None:
        return lib.oracle_threshold_eps(float(mol.eps))
    return lib.oracle_threshold_bits(int(mol.bits))


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} failed with status {rc}")


def _points(mol, points):
    pts = mol.points if points is None else points
    return _c(np.asarray(pts).reshape(-1, 3), np.float64)


def ao_vgl(mol, points=None, screened: bool = True,
           nucl_coord=None) -> Tuple[np.ndarray, np.ndarray]:
    """AO vgl [n][5][ao] and the term-wise size of each entry."""
    lib = _load()
    b = _BasisRef(mol, nucl_coord)
    pts = _points(mol, points)
    n = pts.shape[0]
    out = np.zeros((n, 5, b.ao_num))
    mag = np.zeros((n, 5, b.ao_num))
    _check(lib.oracle_ao_vgl(b.ref, threshold(mol, screened), n, _ptr(pts), _ptr(out),
                             _ptr(mag)), "ao_vgl")
    return out, mag


def mo_from_ao(ao: np.ndarray, C: np.ndarray,
               ao_mag: Optional[np.ndarray] = None) -> Tuple[np.ndarray, Optional[np.ndarray]]:
    """Eqs. 5-7 on a given AO tensor [n][5][ao] with C [mo][ao]."""
    lib = _load()
    ao = _c(ao, np.float64)
    C = _c(C, np.float64)
    n, _, na = ao.shape
    nm = C.shape[0]
    out = np.zeros((n, 5, nm))
    mag = None
    am = None
    if ao_mag is not None:
        am = _c(ao_mag, np.float64)
        mag = np.zeros((n, 5, nm))
    _check(lib.oracle_mo_vgl(na, nm, _ptr(C), n, _ptr(ao), _ptr(am), _ptr(out), _ptr(mag)),
           "mo_vgl")
    return out, mag


def mo_vgl(mol, points=None, screened: bool = True, C=None,
           nucl_coord=None) -> Tuple[np.ndarray, np.ndarray]:
    """MO vgl [n][5][mo] and the term-wise size sum_k |C_nk| size(chi_k)."""
    lib = _load()
    b = _BasisRef(mol, nucl_coord)
    pts = _points(mol, points)
    C = _c(mol.mo_coef if C is None else C, np.float64)
    n = pts.shape[0]
    nm = C.shape[0]
    out = np.zeros((n, 5, nm))
    mag = np.zeros((n, 5, nm))
    _check(lib.oracle_mo_vgl_points(b.ref, threshold(mol, screened), nm, _ptr(C), n,
                                    _ptr(pts), _ptr(out), _ptr(mag)), "mo_vgl_points")
    return out, mag


def adjoint(mol, W: np.ndarray, points=None, screened: bool = True, C=None,
            nucl_coord=None, sizes: bool = False):
    """dL/dC [mo][ao] and dL/dR_nuc [nucl][3] for L = sum W * mo_vgl.

    With sizes=True also returns the term-wise sizes of both sums (the scale
    of their rounding error): (dC, dR, dC_size, dR_size).
    """
    lib = _load()
    b = _BasisRef(mol, nucl_coord)
    pts = _points(mol, points)
    C = _c(mol.mo_coef if C is None else C, np.float64)
    W = _c(W, np.float64)
    n = pts.shape[0]
    nm = C.shape[0]
    if W.shape != (n, 5, nm):
        raise ValueError(f"W has shape {W.shape}, expected {(n, 5, nm)}")
    nn = b.arrs["nucl_coord"].shape[0]
    dC = np.zeros((nm, b.ao_num))
    dR = np.zeros((nn, 3))
    dCs = np.zeros((nm, b.ao_num)) if sizes else None
    dRs = np.zeros((nn, 3)) if sizes else None
    _check(lib.oracle_adjoint(b.ref, threshold(mol, screened), nm, _ptr(C), n, _ptr(pts),
                              _ptr(W), _ptr(dC), _ptr(dR), _ptr(dCs), _ptr(dRs)), "adjoint")
    if sizes:
        return dC, dR, dCs, dRs
    return dC, dR


def screen_counts(mol, points=None, screened: bool = True):
    """(surviving point-shell pairs, evaluated primitives, point-AO pairs)."""
    lib = _load()
    b = _BasisRef(mol)
    pts = _points(mol, points)
    out = np.zeros(3, dtype=np.int64)
    _check(lib.oracle_screen_counts(b.ref, threshold(mol, screened), pts.shape[0], _ptr(pts),
                                    _ptr(out)), "screen_counts")
    return tuple(int(x) for x in out)


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
