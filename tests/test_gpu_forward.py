"""GPU parity of the forward AO/MO vgl path against the FP64 CPU oracle.

Every test calls the CUDA library through its C ABI (ctypes binding) and
compares with the oracle element by element with the normwise metric of
tests/tolerances.py.  Small cases span several tiles and ragged tails in
every dimension; the full organic workload (600 e- x 256 walkers, 300 MOs,
1650 AOs) runs in the benchmark's launch configuration and is checked on
sampled points.
"""
import json
import os

import numpy as np
import pytest

from paper_2512_16677_gb300 import synth
from tolerances import TOL, assert_within, component_errors

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = ["fp64", "fp32", "bf16x3", "tf32"]
REPORT = os.environ.get("QK_PARITY_REPORT")


def _report(name, mode, errs):
    if REPORT:
        with open(REPORT, "a") as f:
            f.write(json.dumps({"case": name, "mode": mode, "value": errs[0],
                                "gradient": errs[1], "laplacian": errs[2]}) + "\n")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_16677_gb300 import buildlib
    buildlib.build()


def _ctx(mol, mode):
    from paper_2512_16677_gb300 import qmckl
    c = qmckl.Context(mode)
    c.set_molecule(mol)
    c.set_points_device(torch.from_numpy(mol.coord).cuda())
    return c


def _run(mol, mode):
    from paper_2512_16677_gb300 import qmckl
    c = _ctx(mol, mode)
    try:
        out = c.mo_vgl_device()
    except qmckl.QmcklError as e:
        if e.status == -5:
            pytest.skip(f"{mode} not built: {e}")
        raise
    torch.cuda.synchronize()
    c.synchronize()
    return c, out.double().cpu().numpy().reshape(-1, 5, mol.mo_num)


@pytest.mark.parametrize("mode", MODES)
def test_water_all_points(orc, cfg, mode):
    """Water: all 640 points, 25 AOs, 5 MOs."""
    m = cfg(1)
    ref, size = orc.mo_vgl(m)
    _, got = _run(m, mode)
    _report("water", mode, assert_within(mode, got, ref, size, "water"))


@pytest.mark.parametrize("mode", ["fp64", "fp32"])
def test_water_ao_vgl(orc, cfg, mode):
    """AO tensor itself (qk_get_ao_vgl_device) against the oracle's AOs."""
    m = cfg(1)
    ref, size = orc.ao_vgl(m)
    c = _ctx(m, mode)
    ao = c.ao_vgl_device()
    torch.cuda.synchronize()
    got = ao.double().cpu().numpy().reshape(ref.shape)
    errs = assert_within(mode, got, ref, size, "water AO")
    _report("water_ao", mode, errs)


@pytest.mark.parametrize("mode", MODES)
def test_chain_two_walkers(orc, cfg, mode):
    """C/H chain, 2 walkers x 200 e- (400 points), 500 AOs, 100 MOs: several
    tiles along points, AOs and MOs, with ragged tails in each."""
    m = cfg(3, walk_num=2)
    ref, size = orc.mo_vgl(m)
    _, got = _run(m, mode)
    _report("chain50_2w", mode, assert_within(mode, got, ref, size, "chain"))


@pytest.mark.parametrize("mode", MODES)
def test_organic_one_walker(orc, cfg, mode):
    """Organic chain, 1 walker (600 points), 1650 AOs up to f, 300 MOs,
    eps = 1e-10 cutoff."""
    m = cfg(2, walk_num=1)
    pts = m.points[::3]          # 200 points, still ragged against every tile
    mm = m.with_points(pts)
    ref, size = orc.mo_vgl(mm)
    _, got = _run(mm, mode)
    _report("organic150_1w", mode, assert_within(mode, got, ref, size, "organic"))


FULL_SAMPLE = 1024     # sampled points of the full organic workload


@pytest.fixture(scope="module")
def organic_full_sample(orc, cfg):
    """The sampled points of the full organic workload (stratified over the
    tiles of the split-bf16 launch) and the oracle's MO vgl at them."""
    from sampling import mo_vgl_threaded, slot_offsets_covered, stratified_points
    m = cfg(2)
    c = _ctx(m, "bf16x3")
    c.mo_vgl_device()
    torch.cuda.synchronize()
    perm, live = c.tile_layout()
    c.close()
    idx = stratified_points(perm, live, FULL_SAMPLE, seed=7)
    assert idx.shape[0] >= FULL_SAMPLE
    assert slot_offsets_covered(perm, idx) == set(range(25))
    ref, size = mo_vgl_threaded(orc, m, m.points[idx])
    return idx, ref, size


@pytest.mark.parametrize("mode", ["bf16x3", "tf32", "fp32", "fp64"])
def test_organic_full_size_sampled(cfg, organic_full_sample, mode):
    """Full benchmark workload (153 600 points) in the benchmark's launch
    configuration, checked on >= 1024 points stratified over tile classes
    (sparsest to densest live-block counts), slot offsets and both ends of
    the permutation."""
    m = cfg(2)
    idx, ref, size = organic_full_sample
    c, got = _run(m, mode)
    errs = assert_within(mode, got[idx], ref, size, "organic full")
    _report("organic150_full_sampled", mode, errs)
    assert np.all(np.isfinite(got))


def test_edge_single_point_and_far_points(orc, cfg):
    """One point; points far from every nucleus give exact zeros."""
    m = cfg(1)
    one = m.with_points(m.points[:1])
    ref, size = orc.mo_vgl(one)
    _, got = _run(one, "fp64")
    assert_within("fp64", got, ref, size, "single point")
    far = m.with_points(np.array([[80.0, 0.0, 0.0], [0.0, -95.0, 3.0], [1e3, 1e3, 1e3]]))
    for mode in MODES:
        _, got = _run(far, mode)
        assert np.all(got == 0.0)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("l, nmo", [(0, 1), (3, 1), (2, 7)])
def test_degenerate_one_shell(orc, mode, l, nmo):
    """One nucleus carrying one shell (1, 10 or 6 AOs: K far below one 64-AO
    chunk) and 1 or 7 MOs (N below one 16-wide MMA step); 37 points, so the
    second 25-point tile is ragged, one of them on the nucleus (d = 0)."""
    centre = np.array([0.3, -0.2, 0.1])
    rng = np.random.default_rng(30 + l)
    pts = centre + rng.normal(scale=1.2, size=(37, 3))
    pts[7] = centre
    nao = (l + 1) * (l + 2) // 2
    C = rng.normal(size=(nmo, nao))
    m = synth.tiny_shell(l, [0.4, 2.5, 30.0], [0.5, 0.3, 0.2], centre=tuple(centre),
                         points=pts, mo_coef=C)
    ref, size = orc.mo_vgl(m)
    _, got = _run(m, mode)
    assert got.shape == ref.shape == (37, 5, nmo)
    assert_within(mode, got, ref, size, f"one l={l} shell, {nmo} MOs")


@pytest.mark.parametrize("mode", MODES)
def test_points_on_nuclei(orc, cfg, mode):
    """Electrons exactly at every nucleus of the organic chain (d = 0 for that
    nucleus's shells) followed by ordinary points: 211 points, a ragged tail."""
    m = cfg(2, walk_num=1)
    mm = m.with_points(np.concatenate([m.nucl_coord, m.points[:61]]))
    ref, size = orc.mo_vgl(mm)
    _, got = _run(mm, mode)
    assert_within(mode, got, ref, size, "points on nuclei")


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_sparse_tiles_mixed(orc, cfg, mode):
    """Tensor-core modes skip blocks of screened AOs: a point set where whole
    25-point tiles are far from every nucleus, others near, others mixed."""
    m = cfg(2, walk_num=1)
    near = m.points[:100]
    far = near + np.array([300.0, 0.0, 0.0])
    mixed = np.concatenate([near[:40], far[:60], near[40:90], far[60:73]])
    mm = m.with_points(mixed)
    ref, size = orc.mo_vgl(mm)
    _, got = _run(mm, mode)
    assert np.all(got[40:100] == 0.0)
    assert_within(mode, got, ref, size, "mixed tiles")


def test_transposed_points_and_host_api(orc, cfg):
    """'T' layout and the host-memory calls give the device results."""
    from paper_2512_16677_gb300 import qmckl
    m = cfg(3, walk_num=1)
    c, dev = _run(m, "fp64")
    c2 = qmckl.Context("fp64")
    c2.set_molecule(m)
    c2.set_points(np.ascontiguousarray(m.points.T), transp="T")
    host = c2.mo_vgl()
    np.testing.assert_array_equal(host, dev)
    ao = c2.ao_vgl()
    ref, size = orc.ao_vgl(m)
    assert_within("fp64", ao, ref, size, "host ao")


def test_memoisation_and_time_stamp(cfg):
    """Same time stamp: the AO tensor is reused (one ao_vgl launch); new
    points bump the stamp and the result changes."""
    m = cfg(1)
    c = _ctx(m, "fp32")
    c.set_timing(True)
    a = c.mo_vgl_device().clone()
    b = c.mo_vgl_device().clone()
    torch.cuda.synchronize()
    ms, n = c.get_timing()
    assert n[0] == 1 and n[1] == 2
    assert torch.equal(a, b)
    c.set_points_device(torch.from_numpy(m.coord[::-1].copy()).cuda())
    d = c.mo_vgl_device()
    torch.cuda.synchronize()
    assert not torch.equal(a, d)
    ms, n = c.get_timing()
    assert n[0] == 1


def test_errors_on_device_calls(cfg):
    from paper_2512_16677_gb300 import qmckl
    m = cfg(1, walk_num=1)
    c = _ctx(m, "fp64")
    small = torch.empty(10, dtype=torch.float64, device="cuda")
    with pytest.raises(qmckl.QmcklError) as e:
        c.lib.qk_get_mo_vgl_device(c.h, small.data_ptr(), 10) and \
            c._check(c.lib.qk_get_mo_vgl_device(c.h, small.data_ptr(), 10), "x")
    assert e.value.status == -3
    ws = torch.empty(1024, dtype=torch.uint8, device="cuda")
    c._check(c.lib.qk_set_workspace(c.h, ws.data_ptr(), 1024), "ws")
    with pytest.raises(qmckl.QmcklError) as e:
        out = torch.empty(m.point_num * 5 * m.mo_num, dtype=torch.float64, device="cuda")
        c._check(c.lib.qk_get_mo_vgl_device(c.h, out.data_ptr(), out.numel()), "x")
    assert e.value.status == -3


def test_primitive_order_invariance_gpu(cfg):
    """The library sorts primitives itself: permuted input, same FP64 output."""
    m = cfg(1, walk_num=4)
    rng = np.random.default_rng(8)
    perm, start = [], 0
    for npr in m.shell_prim_num:
        perm.extend((start + rng.permutation(int(npr))).tolist())
        start += int(npr)
    perm = np.array(perm)
    m2 = synth.Molecule(**{**m.__dict__, "exponent": m.exponent[perm],
                           "coefficient": m.coefficient[perm],
                           "prim_factor": m.prim_factor[perm]})
    _, a = _run(m, "fp64")
    _, b = _run(m2, "fp64")
    np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("case", ["water", "chain", "organic"])
def test_bf16x3_fused_matches_two_kernel_path(orc, cfg, case):
    """split-bf16 with AO blocks built inside the contraction kernel
    (qk_set_fusion(1)) and through an AO tensor in HBM (the default) use the
    same arithmetic; both meet the bar against the oracle."""
    m = {"water": cfg(1), "chain": cfg(3, walk_num=2), "organic": cfg(2, walk_num=1)}[case]
    ref, size = orc.mo_vgl(m)
    outs = []
    for fused in (True, False):
        c = _ctx(m, "bf16x3")
        c.set_fusion(fused)
        o = c.mo_vgl_device()
        torch.cuda.synchronize()
        c.synchronize()
        outs.append(o.double().cpu().numpy().reshape(-1, 5, m.mo_num))
        assert_within("bf16x3", outs[-1], ref, size, f"{case} fused={fused}")
    assert np.max(np.abs(outs[0] - outs[1])) <= 1e-6 * np.max(np.abs(outs[1]))


@pytest.mark.parametrize("mode", ["bf16x3", "tf32", "fp32", "fp64"])
def test_host_output_ranges_match_device(cfg, mode):
    """The host-memory MO call evaluates and copies back point ranges in turn
    (19 200 points: two ranges); the result is bit-identical to the device
    call, both when it evaluates the AOs itself and when it reuses them."""
    from paper_2512_16677_gb300 import qmckl
    m = cfg(2, walk_num=32)
    _, dev = _run(m, mode)
    c = qmckl.Context(mode)
    c.set_molecule(m)
    c.set_points(m.points)
    pinned = torch.empty(m.point_num * 5 * m.mo_num, dtype=torch.float64 if mode == "fp64"
                         else torch.float32, pin_memory=True)
    first = c.mo_vgl(pinned.numpy()).copy()
    again = c.mo_vgl(pinned.numpy())          # AO tensor reused from the first call
    np.testing.assert_array_equal(first, dev)
    np.testing.assert_array_equal(again, dev)
    pageable = c.mo_vgl()                     # plain numpy output buffer
    np.testing.assert_array_equal(pageable, dev)


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_spatial_order_same_values_fewer_blocks(orc, cfg, mode):
    """Tiles cut from the spatial order (default) and from the caller's order
    give the same values; on points handed over in an order with no spatial
    locality the spatial order multiplies far fewer blocks."""
    m = cfg(2, walk_num=8)                       # 4 800 points
    rng = np.random.default_rng(11)
    mm = m.with_points(m.points[rng.permutation(m.point_num)])
    outs, live = [], []
    for spatial in (True, False):
        c = _ctx(mm, mode)
        c.set_spatial_order(spatial)
        o = c.mo_vgl_device()
        torch.cuda.synchronize()
        c.synchronize()
        outs.append(o.double().cpu().numpy().reshape(-1, 5, mm.mo_num))
        live.append(c.block_stats()[0])
    np.testing.assert_array_equal(outs[0], outs[1])
    assert live[0] < 0.6 * live[1], live
    idx = np.sort(rng.choice(mm.point_num, 64, replace=False))
    ref, size = orc.mo_vgl(mm, points=mm.points[idx])
    assert_within(mode, outs[0][idx], ref, size, "spatial order")


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_sparsity_stats(orc, cfg, mode):
    """The nonzero (point, AO) count of the AO tensor agrees with the
    oracle's count of AOs that pass Eq. 3 (screening decided in FP32 on the
    device: a few pairs at the threshold may differ), and the live 16-AO
    groups the contraction's k-steps run over lie between the live blocks
    and four times as many."""
    m = cfg(2, walk_num=8)                       # 4 800 points
    c = _ctx(m, mode)
    o = c.mo_vgl_device()
    torch.cuda.synchronize()
    live, total, entries = c.block_stats()
    groups, nnz = c.sparsity_stats()
    ref = orc.screen_counts(m)[2]
    assert abs(nnz - ref) <= max(8, 1e-4 * ref), (nnz, ref)
    assert live <= groups <= 4 * live
    assert nnz <= entries
    assert nnz <= groups * 16 * 25               # 25 points per tile
    got = o.double().cpu().numpy().reshape(-1, 5, m.mo_num)
    idx = np.sort(np.random.default_rng(5).choice(m.point_num, 48, replace=False))
    r, size = orc.mo_vgl(m, points=m.points[idx])
    assert_within(mode, got[idx], r, size, "group-skipping contraction")


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_reused_context_matches_fresh(cfg, mode):
    """Blocks and 16-AO groups that no point of a tile reaches are neither
    written nor read, so a context that evaluated other points before holds
    stale values there: the MOs of a second point set must still equal, bit
    for bit, those of a fresh context (different points light up different
    groups)."""
    m = cfg(2, walk_num=8)
    rng = np.random.default_rng(21)
    first = m.with_points(m.points + rng.normal(scale=2.0, size=m.points.shape))
    second = m.with_points(m.points[rng.permutation(m.point_num)])
    c = _ctx(first, mode)
    c.mo_vgl_device()
    c.set_points_device(torch.from_numpy(second.coord).cuda())
    reused = c.mo_vgl_device()
    torch.cuda.synchronize()
    _, fresh = _run(second, mode)
    np.testing.assert_array_equal(reused.double().cpu().numpy().reshape(fresh.shape), fresh)


def test_kernel_count(cfg):
    """The library counts the kernels it launches for a step (point
    conversion, spatial order, reach pre-pass, ao_vgl, contraction) and
    resets the count when it is read."""
    m = cfg(2, walk_num=8)
    c = _ctx(m, "bf16x3")
    c.mo_vgl_device()
    torch.cuda.synchronize()
    c.kernel_count()
    c.set_points_device(torch.from_numpy(m.coord).cuda())
    c.mo_vgl_device()
    torch.cuda.synchronize()
    n = c.kernel_count()
    assert n == 1 + 8 + 2 + 1, n      # conversion, sort, pre-pass + ao_vgl, contraction
    assert c.kernel_count() == 0


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_sm_pairs_same_values_as_single_sm(orc, cfg, mode):
    """The contraction on pairs of SMs (cta_group::2, the default) and on
    single SMs multiply the same live blocks; the pair's extra k-steps over
    its partner's live groups add exact zeros.  47 tiles (an odd count: the
    last pair has one tile) of the organic chain, against the oracle and
    against each other."""
    from paper_2512_16677_gb300 import qmckl
    m = cfg(2, walk_num=2)
    mm = m.with_points(m.points[:47 * 25 - 3])
    outs = {}
    for pairs in (True, False):
        c = qmckl.Context(mode)
        c.set_molecule(mm)
        c.set_sm_pairs(pairs)
        c.set_points_device(torch.from_numpy(mm.coord).cuda())
        out = c.mo_vgl_device()
        torch.cuda.synchronize()
        c.synchronize()
        outs[pairs] = out.double().cpu().numpy().reshape(-1, 5, mm.mo_num)
        c.close()
    ref, size = orc.mo_vgl(mm)
    assert_within(mode, outs[True], ref, size, "organic pairs")
    diff = np.abs(outs[True] - outs[False]) / (size + 1e-300)
    assert float(diff.max()) <= 1e-6, float(diff.max())


_WIDTH_REF = {}


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
@pytest.mark.parametrize("mo_num", [40, 72, 120, 150, 180, 250])
def test_sm_pairs_every_tile_width(orc, cfg, mode, mo_num):
    """Every MMA N the contraction picks for up to 256 MOs (64, 96, 128,
    160, 192, 256: one N tile) on pairs of SMs: the first mo_num MOs of the
    organic chain on 47 tiles, against the oracle and the single-SM kernel."""
    import dataclasses

    from paper_2512_16677_gb300 import qmckl
    m = cfg(2, walk_num=2)
    mm = m.with_points(m.points[:47 * 25 - 3])
    if "full" not in _WIDTH_REF:
        _WIDTH_REF["full"] = orc.mo_vgl(mm)
    ref_full, size_full = _WIDTH_REF["full"]
    mk = dataclasses.replace(mm, mo_coef=np.ascontiguousarray(mm.mo_coef[:mo_num]))
    ref, size = ref_full[..., :mo_num], size_full[..., :mo_num]
    outs = {}
    for pairs in (True, False):
        c = qmckl.Context(mode)
        c.set_molecule(mk)
        c.set_sm_pairs(pairs)
        c.set_points_device(torch.from_numpy(mk.coord).cuda())
        out = c.mo_vgl_device()
        torch.cuda.synchronize()
        c.synchronize()
        outs[pairs] = out.double().cpu().numpy().reshape(-1, 5, mo_num)
        c.close()
    assert_within(mode, outs[True], ref, size, f"pairs, {mo_num} MOs")
    diff = np.abs(outs[True] - outs[False]) / (size + 1e-300)
    assert float(diff.max()) <= 1e-6, float(diff.max())


def test_spatial_order_is_the_stable_morton_sort(cfg):
    """The device's point order (one radix sort of the cell keys) equals a
    stable sort of the same keys done here: cells of a 32^3 grid over the
    nuclear box +- 4 bohr, from the float coordinates, bits of the three
    cell indices interleaved x, y, z from the lowest."""
    m = cfg(2, walk_num=16)
    c = _ctx(m, "bf16x3")
    c.mo_vgl_device()
    torch.cuda.synchronize()
    perm, _ = c.tile_layout()
    pts = m.points.astype(np.float32)
    lo = (m.nucl_coord.min(axis=0) - 4.0).astype(np.float32)
    hi = (m.nucl_coord.max(axis=0) + 4.0).astype(np.float32)
    inv = (np.float32(32.0) / np.maximum(hi - lo, np.float32(1e-3))).astype(np.float32)
    f = (pts - lo) * inv
    cell = np.where(f <= 0, 0, np.where(f >= 31, 31, np.trunc(f))).astype(np.uint32)
    key = np.zeros(len(pts), dtype=np.uint32)
    for bit in range(5):
        for axis in range(3):
            key |= ((cell[:, axis] >> bit) & 1) << (3 * bit + axis)
    np.testing.assert_array_equal(perm, np.argsort(key, kind="stable"))
