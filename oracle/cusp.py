"""FP64 oracle of the MO cusp correction (Sec. 3.3).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the tests,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs are its only callers.

Sec. 3.3 replaces, inside a sphere of radius rc_A around nucleus A, each MO
by

    phi_i^cusp(r) = phi_i(r) - phi_i^{s_A}(r) + sum_{k=0}^{3} f_k^{(A,i)} rho^k,
    rho = |r - R_A|,

where phi_i^{s_A} is the part of MO i carried by the s-type AOs on A.  The
paper fixes the f_k by continuity of value and gradient at rc_A and by the
electron-nucleus cusp (Kato), which is three conditions for four
coefficients.  The reading taken here adds continuity of the second radial
derivative (so the Laplacian, and with it the local kinetic energy, is
continuous at rc_A):

    p(rc)   = g(rc)          p(rho) = sum_k f_k rho^k
    p'(rc)  = g'(rc)         g(rho) = phi_i^{s_A} as a function of rho
    p''(rc) = g''(rc)
    f_1     = -Z_A (q + f_0),  q = phi_i(R_A) - g(0)

The last line is Kato's condition on the spherical average of phi^cusp at
the nucleus: everything but g and p is smooth at R_A, so its spherical
average has zero slope there, the average of phi^cusp is q + p(rho) to first
order, and Kato asks its slope f_1 to equal -Z_A times its value q + f_0.

g is the s-part exactly as the MO evaluation forms it, with the same Eq. 3
screening of primitives, so that phi - phi^{s_A} holds no s_A contribution.
Points with rho < rc_A (strict) are corrected; the correction of several
nuclei adds up when spheres overlap.  A point exactly on a nucleus has an
infinite Laplacian (2 f_1 / rho), like the true wave function's.
"""
from __future__ import annotations

import math
from typing import Optional, Tuple

import numpy as np

from . import oracle


def _s_shells(mol, A: int):
    """(shell index, its single AO index) of every s shell on nucleus A."""
    ao0 = np.concatenate([[0], np.cumsum((mol.shell_ang_mom + 1) * (mol.shell_ang_mom + 2) // 2)])
    p0 = np.concatenate([[0], np.cumsum(mol.shell_prim_num)])
    out = []
    for s in range(mol.shell_num):
        if int(mol.shell_nucleus[s]) == A and int(mol.shell_ang_mom[s]) == 0:
            out.append((s, int(ao0[s]), int(p0[s]), int(p0[s + 1])))
    return out


def s_radial(mol, A: int, rho: np.ndarray, T: float) -> np.ndarray:
    """Radial sums of the s shells of A at distances rho: array [3][shells][n]
    with S_m = sum_k c_k gamma_k^m exp(-gamma_k rho^2) (m = 0, 1, 2), c_k =
    N_s a_k f_k, over primitives with gamma_k rho^2 < T (Eq. 3)."""
    rho = np.atleast_1d(np.asarray(rho, dtype=np.float64))
    sh = _s_shells(mol, A)
    S = np.zeros((3, len(sh), rho.size))
    r2 = rho * rho
    for j, (s, _, a, b) in enumerate(sh):
        for k in range(a, b):
            g = float(mol.exponent[k])
            c = float(mol.shell_factor[s] * mol.coefficient[k] * mol.prim_factor[k])
            t = g * r2
            e = np.where(t < T, np.exp(-t), 0.0)
            S[0, j] += c * e
            S[1, j] += c * g * e
            S[2, j] += c * g * g * e
    return S


def s_part(mol, A: int, rho, C: np.ndarray, T: float):
    """g_i(rho), g_i'(rho), g_i''(rho) for every MO i: arrays [mo][n].

    For an s AO, chi = M S_0(rho), d chi/d rho = -2 rho M S_1 and
    d^2 chi/d rho^2 = M (4 rho^2 S_2 - 2 S_1)."""
    rho = np.atleast_1d(np.asarray(rho, dtype=np.float64))
    sh = _s_shells(mol, A)
    S = s_radial(mol, A, rho, T)
    nm = C.shape[0]
    g = np.zeros((nm, rho.size))
    g1 = np.zeros((nm, rho.size))
    g2 = np.zeros((nm, rho.size))
    for j, (s, ao, _, _) in enumerate(sh):
        w = C[:, ao] * float(mol.ao_factor[ao])
        g += np.outer(w, S[0, j])
        g1 += np.outer(w, -2.0 * rho * S[1, j])
        g2 += np.outer(w, 4.0 * rho * rho * S[2, j] - 2.0 * S[1, j])
    return g, g1, g2


def coefficients(mol, rc, C: Optional[np.ndarray] = None, screened: bool = True) -> np.ndarray:
    """f [nucl][mo][4]; zero rows for nuclei with rc_A = 0."""
    C = np.asarray(mol.mo_coef if C is None else C, dtype=np.float64)
    rc = np.asarray(rc, dtype=np.float64)
    T = oracle.threshold(mol, screened)
    nn = mol.nucl_num
    nm = C.shape[0]
    f = np.zeros((nn, nm, 4))
    phiR, _ = oracle.mo_vgl(mol, points=mol.nucl_coord, screened=screened, C=C)
    for A in range(nn):
        r = float(rc[A])
        if r <= 0.0:
            continue
        Z = float(mol.nucl_charge[A])
        g, g1, g2 = s_part(mol, A, np.array([r]), C, T)
        g0, _, _ = s_part(mol, A, np.array([0.0]), C, T)
        q = phiR[A, 0, :] - g0[:, 0]
        M = np.array([[1.0, r, r * r, r ** 3],
                      [0.0, 1.0, 2.0 * r, 3.0 * r * r],
                      [0.0, 0.0, 2.0, 6.0 * r],
                      [Z, 1.0, 0.0, 0.0]])
        rhs = np.stack([g[:, 0], g1[:, 0], g2[:, 0], -Z * q], axis=0)  # [4][mo]
        f[A] = np.linalg.solve(M, rhs).T
    return f


def correction(mol, rc, points, C: Optional[np.ndarray] = None, screened: bool = True,
               f: Optional[np.ndarray] = None) -> Tuple[np.ndarray, np.ndarray]:
    """The added terms [n][5][mo] at the points, and their term-wise size."""
    C = np.asarray(mol.mo_coef if C is None else C, dtype=np.float64)
    rc = np.asarray(rc, dtype=np.float64)
    pts = np.asarray(points, dtype=np.float64).reshape(-1, 3)
    T = oracle.threshold(mol, screened)
    if f is None:
        f = coefficients(mol, rc, C, screened)
    n, nm = pts.shape[0], C.shape[0]
    add = np.zeros((n, 5, nm))
    size = np.zeros((n, 5, nm))
    for A in range(mol.nucl_num):
        r = float(rc[A])
        if r <= 0.0:
            continue
        d = pts - mol.nucl_coord[A][None, :]
        rho = np.sqrt((d * d).sum(1))
        hit = np.nonzero(rho < r)[0]
        if hit.size == 0:
            continue
        rh = rho[hit]
        dh = d[hit]
        sh = _s_shells(mol, A)
        S = s_radial(mol, A, rh, T)
        w = np.stack([C[:, ao] * float(mol.ao_factor[ao]) for (_, ao, _, _) in sh], 1)  # [mo][s]
        G0 = w @ S[0]          # g
        G1 = w @ S[1]          # sum C M S_1
        G2 = w @ S[2]          # sum C M S_2
        fA = f[A]              # [mo][4]
        p = (fA[:, [0]] + fA[:, [1]] * rh + fA[:, [2]] * rh ** 2 + fA[:, [3]] * rh ** 3)
        # d p / d rho divided by rho; d g / d rho divided by rho is -2 G1
        p1r = fA[:, [1]] / rh + 2.0 * fA[:, [2]] + 3.0 * fA[:, [3]] * rh
        lap_p = 2.0 * fA[:, [1]] / rh + 6.0 * fA[:, [2]] + 12.0 * fA[:, [3]] * rh
        lap_g = 4.0 * rh * rh * G2 - 6.0 * G1
        gsc = p1r + 2.0 * G1   # gradient factor multiplying d
        add[hit, 0, :] += (p - G0).T
        for k in range(3):
            add[hit, 1 + k, :] += (gsc * dh[:, k]).T
        add[hit, 4, :] += (lap_p - lap_g).T
        # sizes: magnitudes of the separate terms
        wa = np.abs(w)
        s0 = wa @ np.abs(S[0])
        s1 = wa @ np.abs(S[1])
        s2 = wa @ np.abs(S[2])
        pa = (np.abs(fA[:, [0]]) + np.abs(fA[:, [1]]) * rh + np.abs(fA[:, [2]]) * rh ** 2
              + np.abs(fA[:, [3]]) * rh ** 3)
        p1a = (np.abs(fA[:, [1]]) / rh + 2.0 * np.abs(fA[:, [2]])
               + 3.0 * np.abs(fA[:, [3]]) * rh)
        lpa = (2.0 * np.abs(fA[:, [1]]) / rh + 6.0 * np.abs(fA[:, [2]])
               + 12.0 * np.abs(fA[:, [3]]) * rh)
        size[hit, 0, :] += (pa + s0).T
        for k in range(3):
            size[hit, 1 + k, :] += ((p1a + 2.0 * s1) * np.abs(dh[:, k])).T
        size[hit, 4, :] += (lpa + 4.0 * rh * rh * s2 + 6.0 * s1).T
    return add, size


def mo_vgl_cusp(mol, rc, points=None, C: Optional[np.ndarray] = None,
                screened: bool = True) -> Tuple[np.ndarray, np.ndarray]:
    """Cusp-corrected MO vgl [n][5][mo] and its term-wise size."""
    pts = mol.points if points is None else points
    base, size = oracle.mo_vgl(mol, points=pts, screened=screened, C=C)
    add, asize = correction(mol, rc, pts, C=C, screened=screened)
    return base + add, size + asize
