"""Pins of the density oracle (Sec. 5.4), on the CPU.

* A normalised orbital integrates to its occupation: a single s or d
  Cartesian AO (unit norm by the basis conventions) with weight w gives
  int rho = w on a fine grid.
* The density of two orbitals is the weighted sum of their own densities
  (linear in w, quadratic in each orbital), and never negative.
* Grid order: z runs fastest, then y, then x (cube-file order).
A planted slip (the square replaced by an absolute value) fails the
integral.
"""
import numpy as np
import pytest

from oracle import density as dens
from oracle import oracle as orc
from paper_2512_16677_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def _built():
    orc.build()


def _integral(m, w, half=6.0, n=81):
    h = 2 * half / (n - 1)
    pts = dens.grid_points([-half] * 3, [h] * 3, [n] * 3)
    rho, _ = dens.density(m, w, points=pts, screened=False)
    return rho.sum() * h ** 3


@pytest.mark.parametrize("l, comp", [(0, 0), (2, 1)])
def test_normalised_orbital_integrates_to_its_weight(l, comp):
    m = synth.tiny_shell(l, [0.9, 2.5], [0.7, 0.3])
    nm = m.mo_coef.shape[0]
    w = np.zeros(nm)
    w[comp] = 2.0
    assert abs(_integral(m, w) - 2.0) < 1e-6


def test_linear_in_weights_and_nonnegative():
    m = synth.make_config(1, walk_num=4)
    rng = np.random.default_rng(3)
    w1 = rng.uniform(0, 2, m.mo_num)
    w2 = rng.uniform(0, 2, m.mo_num)
    r1, _ = dens.density(m, w1)
    r2, _ = dens.density(m, w2)
    r12, _ = dens.density(m, w1 + w2)
    assert np.allclose(r12, r1 + r2, rtol=1e-13, atol=0)
    assert np.all(r1 >= 0)
    # one orbital alone: its squared value
    e = np.zeros(m.mo_num)
    e[2] = 1.0
    phi, _ = orc.mo_vgl(m)
    r, _ = dens.density(m, e)
    assert np.array_equal(r, phi[:, 0, 2] ** 2)


def test_grid_order():
    p = dens.grid_points([1.0, 2.0, 3.0], [0.5, 0.25, 0.125], [2, 3, 4])
    assert p.shape == (24, 3)
    assert np.array_equal(p[1], [1.0, 2.0, 3.125])       # z first
    assert np.array_equal(p[4], [1.0, 2.25, 3.0])        # then y
    assert np.array_equal(p[12], [1.5, 2.0, 3.0])        # then x


def test_planted_slip_fails(monkeypatch):
    m = synth.tiny_shell(0, [0.9, 2.5], [0.7, 0.3])
    real = orc.mo_vgl

    def abs_not_square(mol, **kw):
        phi, size = real(mol, **kw)
        return np.sqrt(np.abs(phi)), size

    monkeypatch.setattr(dens.oracle, "mo_vgl", abs_not_square)
    assert abs(_integral(m, np.ones(1)) - 1.0) > 1e-2
