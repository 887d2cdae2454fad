"""Pins of the oracle's adjoint (dL/dC, dL/dR_nuc) for L = sum W * mo_vgl.

The paper's force estimator (Sec. 3.6, Eq. 20) needs nuclear derivatives of
the orbitals up to third order; here they are checked against central finite
differences of the oracle's forward values, and against the translation sum
rule sum_A dL/dR_A = - sum_p dL/dr_p.  Screening makes L discontinuous in the
coordinates, so the finite-difference checks run unscreened.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2512_16677_gb300 import synth


def _loss_from_abar(orc, m, abar, pts, nucl_coord=None):
    ao, _ = orc.ao_vgl(m, points=pts, screened=False, nucl_coord=nucl_coord)
    return math.fsum((abar * ao).ravel())


def test_dC_directional_fd(orc, cfg):
    """L is linear in C, so central differences are exact up to rounding."""
    m = cfg(1)
    rng = np.random.default_rng(20)
    W = synth.random_weights(rng, m.point_num, m.mo_num)
    V = rng.normal(size=m.mo_coef.shape)
    dC, _ = orc.adjoint(m, W)
    h = 1e-5

    def L(C):
        mo, _ = orc.mo_vgl(m, C=C)
        return math.fsum((W * mo).ravel())

    fd = (L(m.mo_coef + h * V) - L(m.mo_coef - h * V)) / (2 * h)
    an = float(np.sum(dC * V))
    assert fd == pytest.approx(an, rel=1e-9)


def test_dC_exact_entries(orc, cfg):
    """A few dL/dC entries against exact rational sums of W * chi."""
    m = cfg(1, walk_num=3)
    rng = np.random.default_rng(21)
    W = synth.random_weights(rng, m.point_num, m.mo_num)
    dC, _ = orc.adjoint(m, W)
    ao, _ = orc.ao_vgl(m)
    for (i, k) in [(0, 0), (2, 7), (4, 24), (1, 13)]:
        ex = sum((Fraction(float(W[p, c, i])) * Fraction(float(ao[p, c, k]))
                  for p in range(m.point_num) for c in range(5)), Fraction(0))
        assert abs(dC[i, k] - float(ex)) <= 4 * np.spacing(abs(float(ex))) + 1e-300


@pytest.mark.parametrize("which", ["water", "chain"])
def test_dR_central_fd(orc, cfg, which):
    """dL/dR_nuc against central differences, h = 1e-5 bohr."""
    if which == "water":
        m = cfg(1)
        pts = m.points[:160]
    else:
        m = cfg(3, walk_num=1)
        pts = m.points[::5]
    rng = np.random.default_rng(22)
    W = synth.random_weights(rng, pts.shape[0], m.mo_num)
    _, dR = orc.adjoint(m, W, points=pts, screened=False)
    abar = np.einsum("pcn,nk->pck", W, m.mo_coef)
    h = 1e-5
    fd = np.zeros_like(dR)
    for A in range(m.nucl_num):
        for j in range(3):
            Rp = m.nucl_coord.copy()
            Rm = m.nucl_coord.copy()
            Rp[A, j] += h
            Rm[A, j] -= h
            fd[A, j] = (_loss_from_abar(orc, m, abar, pts, Rp)
                        - _loss_from_abar(orc, m, abar, pts, Rm)) / (2 * h)
    scale = np.max(np.abs(dR))
    assert np.max(np.abs(fd - dR)) <= 1e-6 * scale


def test_dR_translation_sum_rule(orc, cfg):
    """Moving nuclei and electrons together leaves L unchanged, so
    sum_A dL/dR_A = - sum_p dL/dr_p; dL/dr_p from central differences."""
    m = cfg(1)
    pts = m.points[:60]
    rng = np.random.default_rng(23)
    W = synth.random_weights(rng, pts.shape[0], m.mo_num)
    _, dR = orc.adjoint(m, W, points=pts, screened=False)
    abar = np.einsum("pcn,nk->pck", W, m.mo_coef)
    h = 1e-5
    tot = np.zeros(3)
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        ap, _ = orc.ao_vgl(m, points=pts + e, screened=False)
        am, _ = orc.ao_vgl(m, points=pts - e, screened=False)
        tot[j] = math.fsum(((abar * (ap - am)) / (2 * h)).ravel())
    np.testing.assert_allclose(dR.sum(axis=0), -tot, rtol=1e-6,
                               atol=1e-7 * np.max(np.abs(dR)))


def test_dR_vanishes_for_zero_weights_on_other_nuclei(orc):
    """One shell on nucleus 0 only: every other nucleus gets exactly zero."""
    rng = np.random.default_rng(24)
    pts = rng.normal(size=(30, 3))
    m = synth.tiny_shell(2, [0.5, 3.0], [0.7, 0.4], points=pts)
    m.nucl_charge = np.array([1.0, 1.0])
    m.nucl_coord = np.array([[0.0, 0.0, 0.0], [1.0, 2.0, 3.0]])
    W = synth.random_weights(rng, 30, m.mo_num)
    _, dR = orc.adjoint(m, W, screened=False)
    assert np.all(dR[1] == 0.0) and np.any(dR[0] != 0.0)
