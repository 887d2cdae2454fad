"""Pins of the FP64 cusp-correction oracle (Sec. 3.3), on the CPU.

What the correction must satisfy, checked on the oracle's output rather than
on its formulas:
  * continuity of value, gradient and Laplacian across the sphere rho = rc_A
    (value and gradient are the paper's conditions; the Laplacian is the
    reading that fixes the fourth coefficient);
  * Kato's cusp at the nucleus: the slope of the spherically averaged
    orbital equals -Z_A times its value (the uncorrected Gaussian orbitals
    have zero slope, so this fails without the correction);
  * nothing changes outside the spheres or with all radii zero;
  * with a single s function on the nucleus the corrected orbital inside the
    sphere is a cubic in rho.
Planted mistakes (C^2 row dropped, Kato sign flipped, s part not removed)
must make a pin fail.
"""
import numpy as np
import pytest

from oracle import cusp
from oracle import oracle as orc
from paper_2512_16677_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _unit(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def _corrected(mol, rc, pts, f):
    base, size = orc.mo_vgl(mol, points=pts)
    add, asize = cusp.correction(mol, rc, pts, f=f)
    return base + add, size + asize


def pin_continuity(mol, rc, f, rng, nuclei=None):
    """Value, gradient and Laplacian agree just inside and just outside rc."""
    nuclei = range(mol.nucl_num) if nuclei is None else nuclei
    tol = {0: 1e-5, 1: 1e-4, 2: 1e-4, 3: 1e-4, 4: 1e-3}
    for A in nuclei:
        r = float(rc[A])
        if r <= 0:
            continue
        u = _unit(rng, 3)
        eps = 1e-6 * r
        pin = mol.nucl_coord[A] + (r - eps) * u
        pout = mol.nucl_coord[A] + (r + eps) * u
        vin, sin = _corrected(mol, rc, pin, f)
        vout, sout = _corrected(mol, rc, pout, f)
        for c in range(5):
            scale = np.maximum(np.abs(vin[:, c]).max(axis=0), sin[:, c].max(axis=0)) + 1e-300
            jump = np.abs(vin[:, c] - vout[:, c]).max(axis=0) / scale
            assert jump.max() < tol[c], (A, c, jump.max())


def kato_defect(mol, rc, f, A):
    """Per MO: |slope + Z value| / (|slope| + Z |value|) at the nucleus, from a
    quadratic fit of the 6-point spherical average of the orbital at radii
    h, 2h, 3h, 4h (the fit removes the rho^2 terms from the slope)."""
    r = float(rc[A]) if rc is not None else 0.2
    hs = 1e-6 * r * np.arange(1, 5)
    dirs = np.concatenate([np.eye(3), -np.eye(3)])
    avg = []
    for hh in hs:
        pts = mol.nucl_coord[A] + hh * dirs
        if f is None:
            v, _ = orc.mo_vgl(mol, points=pts)
        else:
            v, _ = _corrected(mol, rc, pts, f)
        avg.append(v[:, 0, :].mean(axis=0))
    coef = np.polyfit(hs, np.array(avg), 2)
    slope, value = coef[1], coef[2]
    Z = float(mol.nucl_charge[A])
    return np.abs(slope + Z * value) / (np.abs(slope) + Z * np.abs(value) + 1e-300)


def pin_kato(mol, rc, f):
    for A in range(mol.nucl_num):
        if rc[A] > 0:
            d = kato_defect(mol, rc, f, A)
            assert d.max() < 1e-5, (A, d.max())


@pytest.fixture(scope="module")
def water():
    orc.build()
    m = synth.make_config(1, walk_num=2)
    rc = synth.cusp_radii(m)
    return m, rc, cusp.coefficients(m, rc)


def test_continuity_at_the_sphere(water):
    m, rc, f = water
    pin_continuity(m, rc, f, np.random.default_rng(1))


def test_kato_cusp_at_each_nucleus(water):
    m, rc, f = water
    pin_kato(m, rc, f)
    # the uncorrected orbitals violate it (zero slope, nonzero value)
    assert min(kato_defect(m, rc, None, A).max() for A in range(m.nucl_num)) > 0.5


def test_unchanged_outside_and_with_zero_radii(water):
    m, rc, f = water
    rng = np.random.default_rng(2)
    far = []
    for A in range(m.nucl_num):
        far.append(m.nucl_coord[A] + (rc[A] * (1.0 + rng.uniform(0.01, 3.0, 8)))[:, None]
                   * _unit(rng, 8))
    far = np.concatenate(far)
    d = np.sqrt(((far[:, None, :] - m.nucl_coord[None]) ** 2).sum(-1))
    far = far[(d >= rc[None, :]).all(1)]
    add, _ = cusp.correction(m, rc, far, f=f)
    assert np.all(add == 0.0)
    base, _ = orc.mo_vgl(m)
    zero = np.zeros(m.nucl_num)
    got, _ = cusp.mo_vgl_cusp(m, zero)
    assert np.array_equal(got, base)


def test_single_s_function_gives_a_cubic_inside():
    orc.build()
    m = synth.tiny_shell(0, [0.8, 3.0], [0.6, 0.4])
    rc = np.array([0.4])
    f = cusp.coefficients(m, rc)
    u = np.array([0.3, -0.5, 0.81])
    u /= np.linalg.norm(u)
    rho = np.array([0.05, 0.12, 0.2, 0.27, 0.33])
    v, _ = _corrected(m, rc, rho[:, None] * u[None, :], f)
    coef = np.polyfit(rho[:4], v[:4, 0, 0], 3)
    assert abs(np.polyval(coef, rho[4]) - v[4, 0, 0]) < 1e-12 * abs(v[4, 0, 0])
    pin_continuity(m, rc, f, np.random.default_rng(3))
    pin_kato(m, rc, f)


def test_chain_molecule_pins():
    """A molecule with several s shells per nucleus and other centres nearby."""
    orc.build()
    m = synth.make_config(3, walk_num=1)
    rc = synth.cusp_radii(m)
    f = cusp.coefficients(m, rc)
    rng = np.random.default_rng(4)
    pin_continuity(m, rc, f, rng, nuclei=[0, 1, 2])
    for A in (0, 1):
        assert kato_defect(m, rc, f, A).max() < 1e-5


# ---- planted mistakes -------------------------------------------------

def _mutant_no_c2(m, rc):
    f = cusp.coefficients(m, rc)
    out = np.zeros_like(f)
    C = m.mo_coef
    T = orc.threshold(m)
    phiR, _ = orc.mo_vgl(m, points=m.nucl_coord)
    for A in range(m.nucl_num):
        r = float(rc[A])
        Z = float(m.nucl_charge[A])
        g, g1, _ = cusp.s_part(m, A, np.array([r]), C, T)
        g0, _, _ = cusp.s_part(m, A, np.array([0.0]), C, T)
        q = phiR[A, 0] - g0[:, 0]
        M = np.array([[1, r, r * r, r ** 3], [0, 1, 2 * r, 3 * r * r], [0, 0, 0, 1.0],
                      [Z, 1, 0, 0]])
        rhs = np.stack([g[:, 0], g1[:, 0], np.zeros_like(q), -Z * q])
        out[A] = np.linalg.solve(M, rhs).T
    return out


def _mutant_kato_sign(m, rc):
    C = m.mo_coef
    T = orc.threshold(m)
    phiR, _ = orc.mo_vgl(m, points=m.nucl_coord)
    out = np.zeros((m.nucl_num, C.shape[0], 4))
    for A in range(m.nucl_num):
        r = float(rc[A])
        Z = float(m.nucl_charge[A])
        g, g1, g2 = cusp.s_part(m, A, np.array([r]), C, T)
        g0, _, _ = cusp.s_part(m, A, np.array([0.0]), C, T)
        q = phiR[A, 0] - g0[:, 0]
        M = np.array([[1, r, r * r, r ** 3], [0, 1, 2 * r, 3 * r * r], [0, 0, 2, 6 * r],
                      [-Z, 1, 0, 0]])
        rhs = np.stack([g[:, 0], g1[:, 0], g2[:, 0], Z * q])
        out[A] = np.linalg.solve(M, rhs).T
    return out


def test_pins_fail_on_dropped_second_derivative(water):
    m, rc, _ = water
    with pytest.raises(AssertionError):
        pin_continuity(m, rc, _mutant_no_c2(m, rc), np.random.default_rng(1))


def test_pins_fail_on_flipped_kato_sign(water):
    m, rc, _ = water
    with pytest.raises(AssertionError):
        pin_kato(m, rc, _mutant_kato_sign(m, rc))


def test_pins_fail_when_s_part_is_kept(water, monkeypatch):
    m, rc, f = water
    real = cusp.s_radial

    def no_subtraction(mol, A, rho, T):
        return real(mol, A, rho, T) * 0.0

    monkeypatch.setattr(cusp, "s_radial", no_subtraction)
    with pytest.raises(AssertionError):
        pin_continuity(m, rc, f, np.random.default_rng(1))
