"""GPU parity of the MO cusp correction (Sec. 3.3) against the FP64 oracle.

Points are placed inside every nucleus's sphere (and outside), so that the
correction is exercised in each mode; the device's FP64 coefficients are
compared with the oracle's, and the host and device calls with each other.
"""
import numpy as np
import pytest

from paper_2512_16677_gb300 import synth
from tolerances import assert_within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = ["fp64", "fp32", "bf16x3", "tf32"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_16677_gb300 import buildlib
    buildlib.build()


@pytest.fixture(scope="module")
def ocusp():
    from oracle import cusp, oracle
    oracle.build()
    return cusp


def _near_points(m, rc, per=6, seed=0):
    """Points inside each sphere (rho in 2%..98% of rc) and just outside."""
    rng = np.random.default_rng(seed)
    out = []
    for A in range(m.nucl_num):
        u = rng.normal(size=(2 * per, 3))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        rho = np.concatenate([rc[A] * rng.uniform(0.02, 0.98, per),
                              rc[A] * rng.uniform(1.01, 1.5, per)])
        out.append(m.nucl_coord[A] + rho[:, None] * u)
    return np.concatenate(out)


def _ctx(m, mode, rc, points):
    from paper_2512_16677_gb300 import qmckl
    c = qmckl.Context(mode)
    c.set_molecule(m)
    c.set_mo_cusp(rc)
    c.set_points_device(torch.from_numpy(np.ascontiguousarray(points)).cuda())
    return c


def _mo(c, n, nm):
    o = c.mo_vgl_device()
    torch.cuda.synchronize()
    c.synchronize()
    return o.double().cpu().numpy().reshape(n, 5, nm)


@pytest.mark.parametrize("case", ["water", "chain"])
def test_coefficients_match_oracle(ocusp, cfg, case):
    m = cfg(1) if case == "water" else cfg(3, walk_num=1)
    rc = synth.cusp_radii(m)
    ref = ocusp.coefficients(m, rc)
    c = _ctx(m, "fp64", rc, m.points[:8])
    got = c.cusp_coefficients_device().cpu().numpy()
    scale = np.abs(ref).max(axis=2, keepdims=True) + 1e-300
    assert np.max(np.abs(got - ref) / scale) < 1e-10


@pytest.mark.parametrize("mode", MODES)
def test_water_points_inside_spheres(ocusp, cfg, mode):
    m = cfg(1)
    rc = synth.cusp_radii(m)
    pts = np.concatenate([_near_points(m, rc), m.points[:64]])
    ref, size = ocusp.mo_vgl_cusp(m, rc, points=pts)
    got = _mo(_ctx(m, mode, rc, pts), pts.shape[0], m.mo_num)
    assert_within(mode, got, ref, size, f"water cusp {mode}")
    # the correction did something: far from the uncorrected values inside
    base, _ = ocusp.oracle.mo_vgl(m, points=pts)
    assert np.max(np.abs(got[:, 0] - base[:, 0])) > 1e-3


@pytest.mark.parametrize("mode", ["bf16x3", "fp64"])
def test_organic_sorted_tiles(ocusp, cfg, mode):
    """Tensor-core tiles in the spatial order: rows land back in the caller's
    order before the correction is added."""
    m = cfg(2, walk_num=1)
    rc = synth.cusp_radii(m)
    rng = np.random.default_rng(5)
    near = _near_points(m, rc, per=1, seed=5)
    pts = np.concatenate([m.points[:400], near])[rng.permutation(400 + near.shape[0])]
    mm = m.with_points(pts)
    idx = np.sort(rng.choice(pts.shape[0], 96, replace=False))
    ref, size = ocusp.mo_vgl_cusp(mm, rc, points=pts[idx])
    got = _mo(_ctx(mm, mode, rc, pts), pts.shape[0], m.mo_num)
    assert_within(mode, got[idx], ref, size, f"organic cusp {mode}")


def test_host_call_equals_device_call(ocusp, cfg):
    from paper_2512_16677_gb300 import qmckl
    m = cfg(2, walk_num=32)          # 19 200 points: the host call works in two ranges
    rc = synth.cusp_radii(m)
    dev = _mo(_ctx(m, "bf16x3", rc, m.points), m.point_num, m.mo_num)
    c = qmckl.Context("bf16x3")
    c.set_molecule(m)
    c.set_mo_cusp(rc)
    c.set_points(m.points)
    host = c.mo_vgl()
    np.testing.assert_array_equal(host, dev)


def test_zero_radii_change_nothing(ocusp, cfg):
    m = cfg(1)
    pts = _near_points(m, synth.cusp_radii(m))
    a = _mo(_ctx(m, "fp64", np.zeros(m.nucl_num), pts), pts.shape[0], m.mo_num)
    from paper_2512_16677_gb300 import qmckl
    c = qmckl.Context("fp64")
    c.set_molecule(m)
    c.set_points_device(torch.from_numpy(pts).cuda())
    b = _mo(c, pts.shape[0], m.mo_num)
    np.testing.assert_array_equal(a, b)


def test_refusals(ocusp, cfg):
    from paper_2512_16677_gb300 import qmckl
    m = cfg(1)
    rc = synth.cusp_radii(m)
    c = _ctx(m, "fp64", rc, m.points)
    W = torch.zeros(m.point_num * 5 * m.mo_num, dtype=torch.float64, device="cuda")
    with pytest.raises(qmckl.QmcklError) as e:
        c.backward_device(W)
    assert e.value.status == -5
    with pytest.raises(qmckl.QmcklError) as e:
        c.set_mo_cusp(-rc)
    assert e.value.status == -1
    c2 = _ctx(m, "bf16x3", rc, m.points)
    with pytest.raises(qmckl.QmcklError) as e:
        qmckl.Batch([c2]).run()
    assert e.value.status == -5
