"""Large system: 1000 nuclei in a 10^4 A^3 cluster, 10 000 Cartesian AOs,
2000 MOs, 4000 e- x 16 walkers, eps = 1e-10: the radial cutoff leaves most
(tile, chunk) blocks empty and the tensor-core path skips them.  Checked
against the FP64 oracle on sampled points in split-bf16 and FP32."""
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
    rng = np.random.default_rng(50)
    idx = np.sort(rng.choice(m.point_num, 10, replace=False))
    idx[-1] = m.point_num - 1
    ref, size = orc.mo_vgl(m, points=m.points[idx])
    assert_within(mode, got[idx].astype(np.float64), ref, size, "cluster1000")
    if mode == "bf16x3":
        live, total, _ = c.block_stats()
        assert 0 < live < total
