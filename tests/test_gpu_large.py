"""Large system: 1000 nuclei in a 10^4 A^3 cluster, 10 000 Cartesian AOs,
2000 MOs, 4000 e- x 16 walkers, eps = 1e-10: the radial cutoff leaves most
(tile, chunk) blocks empty and the tensor-core path skips them.  Checked
against the FP64 oracle on >= 256 sampled points (stratified over the
tiles) in split-bf16 and FP32."""
import numpy as np
import pytest

from tolerances import assert_within

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2512_16677_gb300 import buildlib
    buildlib.build()


@pytest.mark.parametrize("mode", ["bf16x3", "fp32"])
def test_large_cluster_sampled(orc, cfg, mode):
    from paper_2512_16677_gb300 import qmckl
    m = cfg(5)
    assert m.ao_num == 10000 and m.mo_num == 2000 and m.point_num == 64000
    c = qmckl.Context(mode)
    c.set_molecule(m)
    c.set_points_device(torch.from_numpy(m.coord).cuda())
    out = c.mo_vgl_device()
    torch.cuda.synchronize()
    c.synchronize()
    got = out.cpu().numpy().reshape(-1, 5, m.mo_num)
    if mode == "bf16x3":
        live, total, _ = c.block_stats()
        assert 0 < live < total
    _cluster_sample(orc, m, c, mode)
    assert_within(mode, got[_SAMPLE["idx"]].astype(np.float64), _SAMPLE["ref"], _SAMPLE["size"],
                  "cluster1000")


_SAMPLE = {}


def _cluster_sample(orc, m, c, mode):
    """>= 256 points stratified over the split-bf16 launch's tiles (taken
    from the first mode that runs; FP32 alone falls back to its caller order)
    and the oracle at them, computed once for both modes."""
    from sampling import mo_vgl_threaded, stratified_points
    if "idx" in _SAMPLE:
        return
    if mode == "bf16x3":
        perm, live = c.tile_layout()
    else:
        perm = np.arange(m.point_num, dtype=np.int32)
        live = np.zeros((m.point_num + 24) // 25, dtype=np.int32)
    idx = stratified_points(perm, live, 256, seed=50)
    assert idx.shape[0] >= 256
    _SAMPLE["idx"] = idx
    _SAMPLE["ref"], _SAMPLE["size"] = mo_vgl_threaded(orc, m, m.points[idx])


def test_large_cluster_split_bf16_adjoint(orc, cfg):
    """The split-bf16 backward at the cluster's size: 157 AO chunks (three
    32-chunk windows of the mask), 2000 MOs (eight N tiles of 256 in dL/dC^T,
    32 K blocks per Abar item), loss weights on 8 points spread over the
    walkers, against the oracle's adjoint at those points (the bars of the
    split-bf16 adjoint)."""
    from paper_2512_16677_gb300 import qmckl, synth
    m = cfg(5)
    rng = np.random.default_rng(51)
    idx = np.sort(rng.choice(m.point_num, 8, replace=False))
    Wp = synth.random_weights(rng, idx.size, m.mo_num)
    dC, dR, sC, sR = orc.adjoint(m, Wp, points=m.points[idx], sizes=True)
    W = torch.zeros((m.point_num, 5, m.mo_num), dtype=torch.float32)
    W[torch.from_numpy(idx)] = torch.from_numpy(Wp).float()
    c = qmckl.Context("bf16x3")
    c.set_molecule(m)
    c.set_points_device(torch.from_numpy(m.coord).cuda())
    c.mo_vgl_device()
    gC, gR = c.backward_device(W.reshape(m.walk_num, m.elec_num, 5, m.mo_num).cuda())
    torch.cuda.synchronize()
    c.synchronize()
    eC = float(np.max(np.abs(gC.cpu().numpy() - dC) / (sC + 1e-300)))
    eR = float(np.max(np.abs(gR.cpu().numpy() - dR) / (sR + 1e-300)))
    assert eC <= 1e-4, f"dL/dC {eC:.3e}"
    assert eR <= 2e-4, f"dL/dR {eR:.3e}"
