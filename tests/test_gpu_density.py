"""GPU parity of the density on grid points (Sec. 5.4) against the FP64 oracle.

Grids whose point counts are ragged against the 128-point value tiles; all
four modes; occupation weights with zeros; the normwise metric of
tests/tolerances.py on rho with the oracle's size sum_i 2 |w_i phi_i| size(phi_i).
"""
import numpy as np
import pytest

from paper_2512_16677_gb300 import synth
from tolerances import TOL

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
def odens():
    from oracle import density, oracle
    oracle.build()
    return density


def _rho(m, mode, pts, w):
    from paper_2512_16677_gb300 import qmckl
    c = qmckl.Context(mode)
    c.set_molecule(m)
    c.set_points_device(torch.from_numpy(np.ascontiguousarray(pts)).cuda())
    r = c.density_device(w)
    torch.cuda.synchronize()
    c.synchronize()
    return r.double().cpu().numpy()


def _check(mode, got, ref, size, what):
    err = np.abs(got - ref) / (size + 1e-300)
    assert np.all(np.isfinite(got)), what
    assert err.max() <= TOL[mode][0], (what, mode, err.max())


@pytest.mark.parametrize("mode", MODES)
def test_water_grid(odens, cfg, mode):
    m = cfg(1)
    o, h, _ = synth.density_grid(m, n=21)
    pts = odens.grid_points(o, h, (21, 21, 21))          # 9261 points
    w = synth.occupations(m)
    ref, size = odens.density(m, w, points=pts)
    got = _rho(m, mode, pts, w)
    _check(mode, got, ref, size, "water grid")


@pytest.mark.parametrize("mode", MODES)
def test_peptide_standin_sampled(odens, cfg, mode):
    m = cfg(6)
    o, h, _ = synth.density_grid(m, n=23)
    pts = odens.grid_points(o, h, (23, 23, 23))          # 12 167 points
    rng = np.random.default_rng(6)
    w = synth.occupations(m)
    w[rng.choice(m.mo_num, 40, replace=False)] = 0.0     # some MOs empty
    w[:5] = 1.0                                         # some singly occupied
    got = _rho(m, mode, pts, w)
    idx = np.sort(rng.choice(pts.shape[0], 160, replace=False))
    idx[0], idx[-1] = 0, pts.shape[0] - 1
    ref, size = odens.density(m, w, points=pts[idx])
    _check(mode, got[idx], ref, size, "peptide stand-in")
    assert np.all(got >= -1e-6 * size.max())


def test_zero_weights_give_zero(cfg):
    m = cfg(1, walk_num=4)
    got = _rho(m, "bf16x3", m.points, np.zeros(m.mo_num))
    assert np.all(got == 0.0)
