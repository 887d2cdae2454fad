"""Pins of the FP64 CPU oracle against what the paper's definitions fix.

Each test checks the oracle against something other than itself: closed
forms of single Gaussian primitives, finite differences, numerical
quadrature of the normalisation, the rotational invariant of a shell,
exact rational sums, screening bounds of Eq. 3 and translation invariance.
A plausible slip in the oracle (a dropped term, a wrong sign or index, a
wrong Cartesian order, a transposed operand) fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2512_16677_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _norm_err(a, b, mag):
    return float(np.max(np.abs(a - b) / (mag + 1e-300)))


# ---------------------------------------------------------------- Eq. 3 ---

def test_eq3_thresholds_golden(orc):
    """T = (B-1) ln 2 and ln(1/eps), values in tests/golden (Eq. 3)."""
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "eq3_thresholds.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows
    for kind, val, thr in rows:
        m = synth.tiny_shell(0, [1.0], [1.0])
        if kind == "bits":
            m.bits, m.eps = int(val), None
        else:
            m.bits, m.eps = None, float(val)
        assert orc.threshold(m) == pytest.approx(float(thr), rel=1e-15)


# ---------------------------------------------------------- closed forms ---

def _pts(rng, n, scale):
    return rng.normal(scale=scale, size=(n, 3))


@pytest.mark.parametrize("gamma", [0.15, 1.7, 40.0, 2000.0])
def test_closed_form_s(orc, gamma):
    """1-primitive s shell: chi = (2g/pi)^(3/4) e^{-g r^2}, grad = -2 g d chi,
    lap = (4 g^2 r^2 - 6 g) chi (Eqs. 1, 2)."""
    rng = np.random.default_rng(1)
    pts = _pts(rng, 50, 1.0 / math.sqrt(gamma))
    m = synth.tiny_shell(0, [gamma], [0.37], centre=(0.3, -0.2, 0.1), points=pts)
    ao, _ = orc.ao_vgl(m, screened=False)
    d = pts - np.array([0.3, -0.2, 0.1])
    r2 = np.sum(d * d, axis=1)
    chi = (2 * gamma / math.pi) ** 0.75 * np.exp(-gamma * r2)
    np.testing.assert_allclose(ao[:, 0, 0], chi, rtol=1e-13, atol=0)
    for j in range(3):
        np.testing.assert_allclose(ao[:, 1 + j, 0], -2 * gamma * d[:, j] * chi,
                                   rtol=1e-12, atol=1e-14 * gamma * np.max(chi))
    lap = (4 * gamma ** 2 * r2 - 6 * gamma) * chi
    np.testing.assert_allclose(ao[:, 4, 0], lap, rtol=1e-11,
                               atol=1e-13 * gamma * np.max(chi))


def test_closed_form_p_and_d(orc):
    """p and d shells of one primitive: component order x, y, z and
    xx, xy, xz, yy, yz, zz; derivatives worked out by hand."""
    g = 0.8
    rng = np.random.default_rng(2)
    pts = _pts(rng, 40, 1.2)
    n1 = (2 * g / math.pi) ** 0.75 * (4 * g) ** 0.5          # x^1 norm
    mp = synth.tiny_shell(1, [g], [0.5], points=pts)
    ao, _ = orc.ao_vgl(mp, screened=False)
    x, y, z = pts.T
    r2 = x * x + y * y + z * z
    e = np.exp(-g * r2)
    for comp, q in enumerate((x, y, z)):
        np.testing.assert_allclose(ao[:, 0, comp], n1 * q * e, rtol=1e-13)
    # chi_x: d/dx = n(1 - 2 g x^2) e ; d/dy = -2 g x y n e ; lap = n x (4g^2 r^2 - 10 g) e
    tol = dict(rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(ao[:, 1, 0], n1 * (1 - 2 * g * x * x) * e, **tol)
    np.testing.assert_allclose(ao[:, 2, 0], -2 * g * x * y * n1 * e, **tol)
    np.testing.assert_allclose(ao[:, 3, 0], -2 * g * x * z * n1 * e, **tol)
    np.testing.assert_allclose(ao[:, 4, 0], n1 * x * (4 * g * g * r2 - 10 * g) * e, **tol)

    n2 = (2 * g / math.pi) ** 0.75 * (4 * g) / math.sqrt(3.0)  # x^2 norm; M_n = 1 for xx
    md = synth.tiny_shell(2, [g], [0.5], points=pts)
    ao, _ = orc.ao_vgl(md, screened=False)
    mxy = math.sqrt(3.0)                                 # M for (1,1,0): sqrt(3!!/1)
    monos = [x * x, x * y, x * z, y * y, y * z, z * z]
    ms = [1, mxy, mxy, 1, mxy, 1]
    for comp in range(6):
        np.testing.assert_allclose(ao[:, 0, comp], ms[comp] * n2 * monos[comp] * e, rtol=1e-13)
    # lap(xy e) = xy (4g^2 r^2 - 14 g) e ; lap(x^2 e) = (2 - 8 g x^2 + (4 g^2 r^2 - 6 g) x^2) e
    np.testing.assert_allclose(ao[:, 4, 1], mxy * n2 * x * y * (4 * g * g * r2 - 14 * g) * e,
                               rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(
        ao[:, 4, 0], n2 * (2 - 8 * g * x * x + (4 * g * g * r2 - 6 * g) * x * x) * e,
        rtol=1e-10, atol=1e-14)
    # d/dz of xz: (x - 2 g x z^2) e
    np.testing.assert_allclose(ao[:, 3, 2], mxy * n2 * (x - 2 * g * x * z * z) * e,
                               rtol=1e-11, atol=1e-14)


def test_f_shell_value_and_order(orc):
    """f shell component order xxx, xxy, xxz, xyy, xyz, xzz, yyy, yyz, yzz, zzz."""
    g = 1.3
    pts = np.array([[0.3, -0.7, 0.45], [1.1, 0.2, -0.35]])
    m = synth.tiny_shell(3, [g], [1.0], points=pts)
    ao, _ = orc.ao_vgl(m, screened=False)
    x, y, z = pts.T
    e = np.exp(-g * (x * x + y * y + z * z))
    n3 = (2 * g / math.pi) ** 0.75 * (4 * g) ** 1.5 / math.sqrt(15.0)
    powers = [(3, 0, 0), (2, 1, 0), (2, 0, 1), (1, 2, 0), (1, 1, 1), (1, 0, 2),
              (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)]
    df = {0: 1, 1: 1, 2: 3, 3: 15}                      # (2a-1)!!
    for comp, (a, b, c) in enumerate(powers):
        mfac = math.sqrt(15.0 / (df[a] * df[b] * df[c]))
        np.testing.assert_allclose(ao[:, 0, comp], mfac * n3 * x ** a * y ** b * z ** c * e,
                                   rtol=1e-13)


# ---------------------------------------------------- finite differences ---

def test_finite_differences_water(orc, cfg):
    """Gradient and Laplacian of every AO of the water basis against
    4th-order central differences of the values (h = 1e-4 bohr)."""
    m = cfg(1)
    rng = np.random.default_rng(3)
    pts = m.points[rng.choice(m.point_num, 100, replace=False)]
    h = 1e-4
    ao, mag = orc.ao_vgl(m, points=pts, screened=False)

    def val(p):
        return orc.ao_vgl(m, points=p, screened=False)[0][:, 0, :]

    lap = np.zeros_like(ao[:, 0, :])
    f0 = ao[:, 0, :]
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fp1, fm1, fp2, fm2 = val(pts + e), val(pts - e), val(pts + 2 * e), val(pts - 2 * e)
        grad = (fm2 - 8 * fm1 + 8 * fp1 - fp2) / (12 * h)
        assert _norm_err(grad, ao[:, 1 + j, :], mag[:, 1 + j, :]) < 1e-6
        lap += (-fp2 + 16 * fp1 - 30 * f0 + 16 * fm1 - fm2) / (12 * h * h)
    assert _norm_err(lap, ao[:, 4, :], mag[:, 4, :]) < 1e-5


# ------------------------------------------------ normalisation quadrature --

def _sphere_rule(l, nrad=2400, rmin=1e-7, rmax=60.0):
    """Product rule in spherical coordinates: trapezoid in t = ln r, Gauss-Legendre
    in cos(theta), trapezoid in phi.  Exact in the angles for degree <= 2l."""
    t = np.linspace(math.log(rmin), math.log(rmax), nrad)
    dt = t[1] - t[0]
    r = np.exp(t)
    wr = np.full(nrad, dt) * r ** 3            # r^2 dr = r^3 dt
    wr[0] *= 0.5
    wr[-1] *= 0.5
    u, wu = np.polynomial.legendre.leggauss(l + 3)
    nphi = 2 * l + 4
    phi = 2 * math.pi * np.arange(nphi) / nphi
    wphi = np.full(nphi, 2 * math.pi / nphi)
    st = np.sqrt(1 - u * u)
    dirs = np.stack([(st[:, None] * np.cos(phi)[None, :]).ravel(),
                     (st[:, None] * np.sin(phi)[None, :]).ravel(),
                     np.repeat(u, nphi)], axis=1)
    wang = (wu[:, None] * wphi[None, :]).ravel()
    pts = (r[:, None, None] * dirs[None, :, :]).reshape(-1, 3)
    w = (wr[:, None] * wang[None, :]).ravel()
    return pts, w


@pytest.mark.parametrize("l,gammas,coefs", [
    (0, [0.3], [1.0]),
    (0, [0.2, 3.5, 80.0], [0.4, 0.9, 0.3]),
    (1, [0.5, 12.0], [0.8, 0.2]),
    (2, [0.12, 1.5, 30.0], [0.3, 0.6, 0.5]),
    (3, [0.7, 4.0], [0.9, 0.4]),
])
def test_normalisation_quadrature(orc, l, gammas, coefs):
    """Every Cartesian AO of a normalised shell integrates chi^2 to 1
    (the paper's basis check by numerical overlap, Sec. 5.3)."""
    pts, w = _sphere_rule(l)
    m = synth.tiny_shell(l, gammas, coefs, points=pts)
    ao, _ = orc.ao_vgl(m, screened=False)
    norms = np.einsum("p,pk->k", w, ao[:, 0, :] ** 2)
    np.testing.assert_allclose(norms, 1.0, rtol=1e-10)
    # the AOs of one shell are not mutually orthogonal, but the overlap of
    # x^2 and y^2 of a d shell is 1/3 of their norm (angular integral ratio)
    if l == 2:
        ov = np.einsum("p,p->", w, ao[:, 0, 0] * ao[:, 0, 3])
        assert ov == pytest.approx(1.0 / 3.0, rel=1e-10)


@pytest.mark.parametrize("l", [0, 1, 2, 3])
def test_normalisation_gauss_hermite(orc, l):
    """One primitive: chi^2 = poly * e^{-2 g r^2}, integrated exactly by a
    scaled Gauss-Hermite product rule."""
    g = 0.9
    x, wx = np.polynomial.hermite.hermgauss(l + 3)
    s = 1.0 / math.sqrt(2 * g)
    X, Y, Z = np.meshgrid(x * s, x * s, x * s, indexing="ij")
    WX = (wx[:, None, None] * wx[None, :, None] * wx[None, None, :]) * s ** 3
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    m = synth.tiny_shell(l, [g], [0.6], points=pts)
    ao, _ = orc.ao_vgl(m, screened=False)
    wgt = WX.ravel() * np.exp(2 * g * np.sum(pts * pts, axis=1))
    norms = np.einsum("p,pk->k", wgt, ao[:, 0, :] ** 2)
    np.testing.assert_allclose(norms, 1.0, rtol=1e-12)


def test_normalisation_trapezoid_grid(orc):
    """Brute 3-D trapezoid grid on a soft 2-primitive p shell."""
    h = 0.12
    ax = np.arange(-9.0, 9.0 + h / 2, h)
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    m = synth.tiny_shell(1, [0.4, 1.1], [0.5, 0.7], points=pts)
    ao, _ = orc.ao_vgl(m, screened=False)
    norms = np.sum(ao[:, 0, :] ** 2, axis=0) * h ** 3
    np.testing.assert_allclose(norms, 1.0, rtol=1e-6)


# --------------------------------------------------- rotational invariant ---

@pytest.mark.parametrize("l", [1, 2, 3])
def test_rotational_invariant(orc, l):
    """sum_{a+b+c=l} l!/(a!b!c!) (chi_abc/M_abc)^2 = (R_s(r) r^l)^2 depends on
    |r - R_A| only: equal under 20 random rotations of r - R_A."""
    rng = np.random.default_rng(10 + l)
    centre = np.array([0.4, -1.0, 2.0])
    gam = [0.3, 2.0, 9.0]
    cof = [0.5, 0.8, 0.2]
    d0 = rng.normal(size=3) * 0.7
    rots = []
    for _ in range(20):
        q, r = np.linalg.qr(rng.normal(size=(3, 3)))
        rots.append(q * np.sign(np.diag(r)))
    pts = np.array([centre + q @ d0 for q in rots])
    m = synth.tiny_shell(l, gam, cof, centre=tuple(centre), points=pts)
    ao, _ = orc.ao_vgl(m, screened=False)
    pw = synth.cartesian_powers(l)
    mult = np.array([math.factorial(l) / (math.factorial(a) * math.factorial(b) * math.factorial(c))
                     for a, b, c in pw])
    inv = np.sum(mult * (ao[:, 0, :] / m.ao_factor) ** 2, axis=1)
    np.testing.assert_allclose(inv, inv[0], rtol=1e-13)
    # and it equals (R(r) r^l)^2 from the shell data
    r2 = float(d0 @ d0)
    R = m.shell_factor[0] * np.sum(m.coefficient * m.prim_factor * np.exp(-m.exponent * r2))
    assert inv[0] == pytest.approx((R * r2 ** (l / 2)) ** 2, rel=1e-13)


# --------------------------------------------------- MO sums, brute force ---

def _exact_dot(c, a):
    return float(sum((Fraction(float(x)) * Fraction(float(y)) for x, y in zip(c, a)),
                     Fraction(0)))


def test_mo_brute_force_water(orc, cfg):
    """Every MO entry of the water workload against exact rational sums of
    the oracle's own AO values (Eqs. 5-7): within 2 ulp."""
    m = cfg(1)
    ao, mag = orc.ao_vgl(m)
    mo, _ = orc.mo_from_ao(ao, m.mo_coef, mag)
    rng = np.random.default_rng(4)
    for p in rng.choice(m.point_num, 60, replace=False):
        for c in range(5):
            for n in range(m.mo_num):
                ex = _exact_dot(m.mo_coef[n], ao[p, c])
                assert abs(mo[p, c, n] - ex) <= 2 * np.spacing(abs(ex)) + 1e-300


_SPLIT = 134217729.0  # 2^27 + 1: Dekker's splitting constant for FP64


def _two_product(x, y):
    """x * y = p + e exactly (Dekker 1971, Veltkamp splitting), elementwise;
    exact unless a product under- or overflows."""
    p = x * y
    cx = _SPLIT * x
    xh = cx - (cx - x)
    xl = x - xh
    cy = _SPLIT * y
    yh = cy - (cy - y)
    yl = y - yh
    e = ((xh * yh - p) + xh * yl + xl * yh) + xl * yl
    return p, e


def _exact_mo(C, ao):
    """Correctly rounded sum_k C[n,k] ao[c,k] for every (c, n) of one point:
    the products split exactly into p + e, then math.fsum (Shewchuk), which
    rounds the exact sum of its arguments once."""
    p, e = _two_product(C[None, :, :], ao[:, None, :])        # [5][mo][ao]
    terms = np.concatenate([p, e], axis=-1).reshape(-1, 2 * C.shape[1]).tolist()
    return np.array([math.fsum(t) for t in terms]).reshape(5, C.shape[0])


@pytest.mark.parametrize("which, walk_num, npts, nmo", [
    (1, None, None, None),   # water, every point
    (3, 1, 48, None),        # 50-nucleus chain, 500 AOs
    (2, 1, 12, None),        # organic chain, 1650 AOs, 300 MOs
    (5, 1, 2, 48),           # 1000-nucleus cluster, 10 000 AOs (48 of the MOs)
])
def test_mo_brute_force_sums(orc, cfg, which, walk_num, npts, nmo):
    """The oracle's MO sums (Eqs. 5-7, compensated Dot2) against correctly
    rounded exact sums of the same AO values, on whole small workloads and
    sampled points of large ones: within the Ogita-Rump-Oishi bound
    eps|s| + 2 (K eps)^2 sum|C chi| (K AOs per sum)."""
    m = cfg(which, walk_num=walk_num)
    pts = m.points
    if npts is not None:
        idx = np.random.default_rng(11).choice(m.point_num, npts, replace=False)
        pts = m.points[np.sort(idx)]
    C = m.mo_coef if nmo is None else m.mo_coef[:nmo]
    ao, _ = orc.ao_vgl(m, points=pts)
    mo, _ = orc.mo_from_ao(ao, C)
    eps = 2.0 ** -53
    K = C.shape[1]
    live = 0
    for q in range(len(pts)):
        ex = _exact_mo(C, ao[q])
        size = np.abs(ao[q])[:, None, :] * np.abs(C)[None, :, :]
        bound = eps * np.abs(ex) + 2 * (K * eps) ** 2 * size.sum(-1)
        assert np.all(np.abs(mo[q] - ex) <= bound), (which, q)
        live += int(np.count_nonzero(ex))
    assert live > 0


def test_mo_layout_and_transpose(orc, cfg):
    """Non-square C: output [point][component][mo] = C @ ao (not C^T)."""
    m = cfg(3, walk_num=1)
    pts = m.points[:7]
    mo, _ = orc.mo_vgl(m, points=pts)
    ao, _ = orc.ao_vgl(m, points=pts)
    ref = np.einsum("nk,pck->pcn", m.mo_coef, ao)
    scale = np.einsum("nk,pck->pcn", np.abs(m.mo_coef), np.abs(ao))
    assert _norm_err(mo, ref, scale) < 1e-13


def test_dot2_ill_conditioned(orc):
    """Dot2 on sums with heavy cancellation stays at the Ogita-Rump-Oishi
    bound eps|s| + 2 (n eps)^2 sum|x y| (a plain sum would not)."""
    rng = np.random.default_rng(5)
    n = 400
    for trial in range(20):
        x = rng.normal(size=n) * np.exp(rng.uniform(-20, 20, size=n))
        y = rng.normal(size=n)
        # force cancellation: append the negated partial sum split into pieces
        s = float(np.dot(x, y))
        x = np.concatenate([x, [-s, s * 1e-17, 1.0]])
        y = np.concatenate([y, [1.0, 1.0, 1e-30]])
        ex = _exact_dot(y, x)
        ao = x.reshape(1, 1, -1).repeat(5, axis=1)
        mo, _ = orc.mo_from_ao(ao, y.reshape(1, -1))
        eps = 2.0 ** -53
        bound = eps * abs(ex) + 2 * (len(x) * eps) ** 2 * float(np.sum(np.abs(x * y)))
        assert abs(mo[0, 0, 0] - ex) <= bound


# ------------------------------------------------------------- screening ---

def test_screening_bound(orc, cfg):
    """Screened minus unscreened is bounded by the dropped primitives,
    each below e^{-T} times its own size (Eq. 3)."""
    m = cfg(2, walk_num=1)
    pts = m.points[:40]
    s, smag = orc.ao_vgl(m, points=pts)
    u, mag = orc.ao_vgl(m, points=pts, screened=False)
    T = orc.threshold(m)
    assert np.any(s != u)       # something was screened
    # (1) the difference is at most the size of the dropped terms
    dropped = mag - smag
    assert np.all(dropped >= -1e-15 * mag)
    assert np.all(np.abs(s - u) <= dropped * (1 + 1e-12) + 1e-15 * mag + 1e-300)
    # (2) value component: each dropped primitive is below e^{-T} times
    #     |M_n N_s a_k f_k P(r)|, summed over the shell's primitives
    ao0 = 0
    p0 = 0
    for sh in range(m.shell_num):
        l = int(m.shell_ang_mom[sh])
        npr = int(m.shell_prim_num[sh])
        d = pts - m.nucl_coord[m.shell_nucleus[sh]]
        cf = np.sum(np.abs(m.coefficient[p0:p0 + npr] * m.prim_factor[p0:p0 + npr]))
        for j, (a, b, c) in enumerate(synth.cartesian_powers(l)):
            P = np.abs(d[:, 0] ** a * d[:, 1] ** b * d[:, 2] ** c)
            bound = math.exp(-T) * m.ao_factor[ao0 + j] * m.shell_factor[sh] * cf * P
            assert np.all(np.abs(s[:, 0, ao0 + j] - u[:, 0, ao0 + j]) <= bound * (1 + 1e-9))
        ao0 += (l + 1) * (l + 2) // 2
        p0 += npr
    # (3) MO level: through |C|
    ms, msmag = orc.mo_vgl(m, points=pts)
    mu, mmag = orc.mo_vgl(m, points=pts, screened=False)
    assert np.all(np.abs(ms - mu) <= (mmag - msmag) * (1 + 1e-9) + 1e-15 * mmag)


def test_screening_all_or_nothing(orc):
    """Far from the nucleus every primitive is screened -> exact zeros; the
    threshold is strict (gamma r^2 < T evaluates)."""
    g = 2.0
    T = orc.threshold(synth.tiny_shell(0, [g], [1.0]))
    r_edge = math.sqrt(T / g)
    pts = np.array([[r_edge * 1.001, 0, 0], [r_edge * 0.999, 0, 0], [0, 0, 50.0]])
    m = synth.tiny_shell(1, [g], [1.0], points=pts)
    ao, _ = orc.ao_vgl(m)
    assert np.all(ao[0] == 0.0) and np.all(ao[2] == 0.0)
    assert np.all(ao[1, 0, :1] != 0.0)


def test_primitive_order_invariance(orc, cfg):
    """Permuting primitives inside each shell changes only rounding."""
    m = cfg(1, walk_num=2)
    rng = np.random.default_rng(6)
    perm = []
    start = 0
    for npr in m.shell_prim_num:
        perm.extend((start + rng.permutation(int(npr))).tolist())
        start += int(npr)
    perm = np.array(perm)
    m2 = synth.Molecule(**{**m.__dict__, "exponent": m.exponent[perm],
                           "coefficient": m.coefficient[perm],
                           "prim_factor": m.prim_factor[perm]})
    a, mag = orc.ao_vgl(m)
    b, _ = orc.ao_vgl(m2)
    assert _norm_err(a, b, mag) < 1e-14


def test_translation_invariance(orc, cfg):
    """Shifting nuclei and points together leaves the AOs unchanged up to the
    rounding of the coordinate differences."""
    m = cfg(1, walk_num=4)
    shift = np.array([7.5, -3.25, 5.0])
    a, mag = orc.ao_vgl(m)
    mt = synth.Molecule(**{**m.__dict__, "nucl_coord": m.nucl_coord + shift,
                           "coord": m.coord + shift})
    b, _ = orc.ao_vgl(mt)
    assert _norm_err(a, b, mag) < 1e-11


def test_screen_counts_match_tables(orc, cfg):
    """screen_counts agrees with the zero pattern of the screened AO tensor."""
    m = cfg(1, walk_num=3)
    pairs, prims, aos = orc.screen_counts(m)
    ao, _ = orc.ao_vgl(m)
    nz = np.any(ao != 0.0, axis=1)       # [point][ao]
    assert aos >= int(nz.sum())
    assert 0 < pairs <= m.point_num * m.shell_num
    assert pairs <= prims <= m.point_num * m.prim_num


def _screen_pin_molecule(bits, eps):
    """Two nuclei 10 bohr apart on x: an s shell (gamma 0.1, 1, 10) and a p
    shell (0.5, 4) on A at the origin, a d shell (2) on B; seven points whose
    squared distances to A and B are whole numbers (or 18.9^2)."""
    g = np.array([0.1, 1.0, 10.0, 0.5, 4.0, 2.0])
    pts = np.array([[1, 0, 0], [3, 0, 0], [5, 0, 0], [8, 0, 0], [10, 0, 0], [30, 0, 0],
                    [0, 18.9, 0]], dtype=float)
    return synth.Molecule(
        "screen-pin", np.array([1.0, 1.0]), np.array([[0, 0, 0], [10, 0, 0]], dtype=float),
        np.array([0, 0, 1], dtype=np.int64), np.array([0, 1, 2], dtype=np.int32),
        np.array([3, 2, 1], dtype=np.int64), np.ones(3), g, np.ones(6), np.ones(6),
        np.ones(10), np.eye(10), pts.reshape(1, -1, 3), bits=bits, eps=eps)


# (surviving point-shell pairs, evaluated primitives, point-AO pairs) per
# point, counted by hand from gamma r^2 < T (Eq. 3):
#   B = 53 -> T = 36.04; r^2_A = 1, 9, 25, 64, 100, 900, 357.21 and
#   r^2_B = 81, 49, 25, 4, 0, 400, 457.21.  E.g. at x = 8: s passes 0.1*64,
#   p passes 0.5*64, d passes 2*4 -> 3 shells, 3 primitives, 1 + 3 + 6 AOs;
#   at (0, 18.9, 0) only 0.1 * 357.21 = 35.72 passes.
#   eps = 1e-10 -> T = 23.03: the same points lose 1*25, 0.5*64, 4*9 and
#   0.1*357.21.
_SCREEN_PIN = {
    (53, None): [(2, 5, 4), (2, 4, 4), (2, 3, 4), (3, 3, 10), (2, 2, 7), (0, 0, 0),
                 (1, 1, 1)],
    (None, 1e-10): [(2, 5, 4), (2, 3, 4), (2, 2, 4), (2, 2, 7), (2, 2, 7), (0, 0, 0),
                    (0, 0, 0)],
}


@pytest.mark.parametrize("bits,eps", list(_SCREEN_PIN))
def test_screen_counts_hand_counted(orc, bits, eps):
    """screen_counts equals hand counts of Eq. 3 on a two-nucleus case, point
    by point and in total (the roofline's denominator rests on it)."""
    m = _screen_pin_molecule(bits, eps)
    want = _SCREEN_PIN[(bits, eps)]
    for p, w in zip(m.points, want):
        assert orc.screen_counts(m, points=p[None, :]) == w, p
    assert orc.screen_counts(m) == tuple(int(sum(c)) for c in zip(*want))
