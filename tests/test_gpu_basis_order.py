"""GPU parity with the shells run in the library's spatial (Morton) order:
every output keeps the caller's AO order (MO vgl, the AO tensor, dL/dC),
the cusp correction and the density see the same basis, and a basis in
random atom order multiplies fewer blocks than in the caller's order."""
import numpy as np
import pytest

from paper_2512_16677_gb300 import synth
from test_basis_order import relist_shells
from tolerances import TOL, assert_within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = ["fp64", "fp32", "bf16x3", "tf32"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_16677_gb300 import buildlib
    buildlib.build()


def _ctx(m, mode, order):
    from paper_2512_16677_gb300 import qmckl
    c = qmckl.Context(mode)
    c.set_basis_order(order)
    c.set_molecule(m)
    c.set_points_device(torch.from_numpy(m.coord).cuda())
    return c


def _shuffled(m, seed=3):
    m2, _ = relist_shells(m, np.random.default_rng(seed).permutation(m.nucl_num))
    return m2


@pytest.mark.parametrize("mode", MODES)
def test_mo_vgl_spatial_order(orc, cfg, mode):
    m = _shuffled(cfg(3, walk_num=2))
    c = _ctx(m, mode, 2)
    assert c.basis_order_spatial()
    got = c.mo_vgl_device()
    torch.cuda.synchronize()
    got = got.double().cpu().numpy().reshape(-1, 5, m.mo_num)
    ref, size = orc.mo_vgl(m)
    assert_within(mode, got, ref, size, f"spatial basis {mode}")


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_ao_tensor_in_caller_columns(orc, cfg, mode):
    m = _shuffled(cfg(1, walk_num=8))
    c = _ctx(m, mode, 2)
    ao = c.ao_vgl_device()
    torch.cuda.synchronize()
    ref, size = orc.ao_vgl(m)
    assert_within(mode, ao.double().cpu().numpy().reshape(ref.shape), ref, size, "AO columns")


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_adjoint_dC_in_caller_columns(orc, cfg, mode):
    m = _shuffled(cfg(3, walk_num=1))
    c = _ctx(m, mode, 2)
    o = c.mo_vgl_device()
    W = torch.from_numpy(np.random.default_rng(4).normal(size=o.shape)).to(o.dtype).cuda()
    dC, dR = c.backward_device(W)
    torch.cuda.synchronize()
    rdC, rdR, sC, sR = orc.adjoint(m, W.double().cpu().numpy().reshape(-1, 5, m.mo_num),
                                   sizes=True)
    bar = 1e-12 if mode == "fp64" else 2e-4
    assert np.max(np.abs(dC.cpu().numpy() - rdC) / (sC + 1e-300)) < bar
    assert np.max(np.abs(dR.cpu().numpy() - rdR) / (sR + 1e-300)) < bar


def test_cusp_and_density_spatial_order(cfg):
    from oracle import cusp, density, oracle
    oracle.build()
    m = _shuffled(cfg(1, walk_num=4))
    rc = synth.cusp_radii(m)
    pts = m.nucl_coord + 0.3 * rc[:, None] * np.array([[0.3, 0.4, 0.866]])
    mm = m.with_points(np.concatenate([pts, m.points[:30]]))
    c = _ctx(mm, "fp64", 2)
    c.set_mo_cusp(rc)
    got = c.mo_vgl_device()
    torch.cuda.synchronize()
    ref, size = cusp.mo_vgl_cusp(mm, rc)
    assert_within("fp64", got.cpu().numpy().reshape(ref.shape), ref, size, "cusp, spatial basis")
    w = synth.occupations(mm)
    rho = c.density_device(w)
    torch.cuda.synchronize()
    rref, rsize = density.density(mm, w)
    assert np.max(np.abs(rho.cpu().numpy() - rref) / (rsize + 1e-300)) < TOL["fp64"][0]


def test_cluster_goes_spatial_with_fewer_blocks(orc, cfg):
    m = cfg(5, walk_num=1)
    live = []
    for order in (0, 1):
        c = _ctx(m, "bf16x3", order)
        assert c.basis_order_spatial() == (order == 0)
        o = c.mo_vgl_device()
        torch.cuda.synchronize()
        live.append(c.block_stats()[0])
        if order == 0:
            got = o.double().cpu().numpy().reshape(-1, 5, m.mo_num)
            idx = np.sort(np.random.default_rng(1).choice(m.point_num, 48, replace=False))
            ref, size = orc.mo_vgl(m, points=m.points[idx])
            assert_within("bf16x3", got[idx], ref, size, "cluster, spatial basis")
    assert live[0] < 0.7 * live[1], live
