"""FP64 oracle of the electron density on grid points (Sec. 5.4).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``.

Sec. 5.4 evaluates the density of a determinant on a Cartesian grid as the
occupation-weighted sum of squared MO values,

    rho(p) = sum_i w_i phi_i(p)^2,

with the MO values of Eqs. 5-7 (value component only).  ``size`` is the
scale the rounding error of rho is measured against:
sum_i w_i 2 |phi_i| size(phi_i), size(phi_i) being the MO oracle's
term-wise size.
"""
from __future__ import annotations

from typing import Tuple

import numpy as np

from . import oracle


def density(mol, w, points=None, screened: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    """rho [n] and its size [n] at the points (default: the molecule's)."""
    w = np.asarray(w, dtype=np.float64)
    if w.shape != (mol.mo_coef.shape[0],):
        raise ValueError("one occupation weight per MO")
    phi, size = oracle.mo_vgl(mol, points=points, screened=screened)
    v = phi[:, 0, :]
    rho = np.array([np.dot(w, vi * vi) for vi in v])
    sz = (2.0 * np.abs(w)[None, :] * np.abs(v) * size[:, 0, :]).sum(axis=1)
    return rho, sz


def grid_points(origin, spacing, n) -> np.ndarray:
    """Points of an n[0] x n[1] x n[2] grid in cube-file order (z fastest)."""
    o = np.asarray(origin, dtype=np.float64)
    h = np.asarray(spacing, dtype=np.float64)
    ix, iy, iz = np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij")
    return np.stack([o[0] + h[0] * ix, o[1] + h[1] * iy, o[2] + h[2] * iz], -1).reshape(-1, 3)
