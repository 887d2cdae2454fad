"""Single-electron moves on the GPU: MO vgl at the proposed positions of one
electron per walker, against the oracle, and against the full evaluation of
the accepted configuration (each row of the MO tensor depends on its own
point only).  The reduced modes run the moved points through the full
path's tile kernels, so the two agree bit for bit; fp64 takes one launch
(each point's AO row and a GEMV against C^T), which agrees within the FP64
bar.  The rows of the other electrons stay bit for bit."""
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


def _ctx(m, mode, cusp=False):
    from paper_2512_16677_gb300 import qmckl
    c = qmckl.Context(mode)
    c.set_molecule(m)
    if cusp:
        c.set_mo_cusp(synth.cusp_radii(m))
    c.set_points_device(torch.from_numpy(m.coord).cuda())
    return c


def _np(t, shape):
    torch.cuda.synchronize()
    return t.double().cpu().numpy().reshape(shape)


def _proposal(m, elec, seed):
    rng = np.random.default_rng(seed)
    return m.coord[:, elec, :] + 0.3 * rng.normal(size=(m.walk_num, 3))


@pytest.mark.parametrize("mode", MODES)
def test_water_single_move(orc, cfg, mode):
    m = cfg(1)
    elec = 3
    new = _proposal(m, elec, 1)
    c = _ctx(m, mode)
    before = _np(c.mo_vgl_device(), (m.walk_num, m.elec_num, 5, m.mo_num))
    c.set_single_point_device(elec, torch.from_numpy(np.ascontiguousarray(new)).cuda())
    single = _np(c.mo_vgl_single_device(), (m.walk_num, 5, m.mo_num))
    ref, size = orc.mo_vgl(m, points=new)
    assert_within(mode, single, ref, size, f"single move {mode}")
    c.accept_single_point()
    after = _np(c.mo_vgl_device(), (m.walk_num, m.elec_num, 5, m.mo_num))
    assert_within(mode, after[:, elec], ref, size, f"accepted move {mode}")
    if mode == "fp64":
        assert_within(mode, single, after[:, elec], size, f"single vs full {mode}")
    else:
        np.testing.assert_array_equal(after[:, elec], single)
    others = [e for e in range(m.elec_num) if e != elec]
    np.testing.assert_array_equal(after[:, others], before[:, others])


@pytest.mark.parametrize("cusp", [False, True])
def test_organic_single_move_matches_full(orc, cfg, cusp):
    m = cfg(2, walk_num=64)
    elec = 417
    new = _proposal(m, elec, 2)
    if cusp:  # put a few proposals inside cusp spheres
        rc = synth.cusp_radii(m)
        new[:4] = m.nucl_coord[:4] + 0.5 * rc[:4, None] * np.array([[0.6, 0.0, 0.8]])
    c = _ctx(m, "bf16x3", cusp=cusp)
    c.mo_vgl_device()
    c.set_single_point_device(elec, torch.from_numpy(np.ascontiguousarray(new)).cuda())
    single = _np(c.mo_vgl_single_device(), (m.walk_num, 5, m.mo_num))
    c.accept_single_point()
    after = _np(c.mo_vgl_device(), (m.walk_num, m.elec_num, 5, m.mo_num))
    if not cusp:
        ref, size = orc.mo_vgl(m, points=new)
    else:  # the corrected MOs (Sec. 3.3) from the cusp oracle
        from oracle import cusp as ocusp
        ref, size = ocusp.mo_vgl_cusp(m, synth.cusp_radii(m), points=new)
    assert_within("bf16x3", single, ref, size, "organic single move")
    assert_within("bf16x3", after[:, elec], ref, size, "organic accepted move")
    np.testing.assert_array_equal(after[:, elec], single)


def test_single_move_errors(cfg):
    from paper_2512_16677_gb300 import qmckl
    m = cfg(1, walk_num=4)
    c = _ctx(m, "fp64")
    with pytest.raises(qmckl.QmcklError) as e:
        c.mo_vgl_single_device()
    assert e.value.status == -4
    with pytest.raises(qmckl.QmcklError) as e:
        c.accept_single_point()
    assert e.value.status == -4
    bad = torch.zeros((m.walk_num, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(qmckl.QmcklError) as e:
        c.set_single_point_device(m.elec_num, bad)
    assert e.value.status == -1


def test_large_basis_fp64_single_move_uses_tile_kernels(orc, cfg):
    """A basis too large for the one-launch FP64 kernel's shared memory (the
    1000-nucleus cluster, 4500 shells) takes the tile kernels; the moved rows
    still match the oracle."""
    m = cfg(5, walk_num=2)
    elec = 1234
    new = _proposal(m, elec, 3)
    c = _ctx(m, "fp64")
    c.mo_vgl_device()
    c.set_single_point_device(elec, torch.from_numpy(np.ascontiguousarray(new)).cuda())
    single = _np(c.mo_vgl_single_device(), (m.walk_num, 5, m.mo_num))
    ref, size = orc.mo_vgl(m, points=new)
    assert_within("fp64", single, ref, size, "cluster single move")
