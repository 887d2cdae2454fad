"""Uneven multi-molecule batch: 12 synthetic chains of 20-200 nuclei, 16-256
walkers, in one persistent ao_vgl launch and one persistent tcgen05 launch
captured in a CUDA graph.  Every molecule is checked against the FP64
oracle on sampled points (stated bf16x3 tolerance), the graph replay must
follow new electron positions, and the autotuned tile must give the same
results."""
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


def _contexts(mols, coords):
    from paper_2512_16677_gb300 import qmckl
    ctxs = []
    for m, c in zip(mols, coords):
        ctx = qmckl.Context("bf16x3")
        ctx.set_molecule(m)
        ctx.set_points_device(c)
        ctxs.append(ctx)
    return ctxs


def _check_all(orc, mols, outs, shift=0.0, n=12, seed=0):
    rng = np.random.default_rng(seed)
    for m, out in zip(mols, outs):
        got = out.double().cpu().numpy().reshape(-1, 5, m.mo_num)
        idx = np.sort(rng.choice(m.point_num, min(n, m.point_num), replace=False))
        idx[-1] = m.point_num - 1
        ref, size = orc.mo_vgl(m, points=m.points[idx] + shift)
        assert_within("bf16x3", got[idx], ref, size, m.name)


def test_uneven_batch_graph_and_autotune(orc, cfg):
    from paper_2512_16677_gb300 import qmckl
    mols = cfg(4)
    assert len(mols) == 12
    assert len({m.ao_num for m in mols}) > 6          # uneven sizes
    coords = [torch.from_numpy(m.coord).cuda() for m in mols]
    ctxs = _contexts(mols, coords)
    b = qmckl.Batch(ctxs)
    outs = b.run()                                    # capture + first replay
    b.synchronize()
    _check_all(orc, mols, outs)
    # new electron positions: same buffers, replayed graph sees them
    shift = 0.05
    for c, x in zip(ctxs, coords):
        c.set_points_device(x + shift)
    outs = b.run()
    b.synchronize()
    _check_all(orc, mols, outs, shift=shift, seed=1)
    # the batch equals one launch per molecule
    for c, m, o in zip(ctxs[:3], mols[:3], outs[:3]):
        single = c.mo_vgl_device()
        torch.cuda.synchronize()
        ref = single.double().cpu().numpy().reshape(-1, 5, m.mo_num)
        got = o.double().cpu().numpy().reshape(-1, 5, m.mo_num)
        scale = np.abs(ref).max()
        assert np.max(np.abs(got - ref)) <= 1e-5 * scale
    bn, ms = b.autotune(reps=2)
    assert bn in (64, 96, 128, 160, 192, 256) and ms > 0
    for c, x in zip(ctxs, coords):
        c.set_points_device(x)
    outs = b.run()
    b.synchronize()
    _check_all(orc, mols, outs, seed=2)


def test_batch_rejects_mixed_or_unset(cfg):
    from paper_2512_16677_gb300 import qmckl
    mols = cfg(4, walk_num=2)[:2]
    a = qmckl.Context("bf16x3")
    a.set_molecule(mols[0])
    a.set_points_device(torch.from_numpy(mols[0].coord).cuda())
    c = qmckl.Context("fp32")
    c.set_molecule(mols[1])
    c.set_points_device(torch.from_numpy(mols[1].coord).cuda())
    with pytest.raises(qmckl.QmcklError):
        qmckl.Batch([a, c])
    d = qmckl.Context("bf16x3")
    d.set_molecule(mols[1])                           # no points
    with pytest.raises(qmckl.QmcklError):
        qmckl.Batch([a, d])


def test_batch_follows_a_cutoff_change(orc, cfg):
    """A context's Eq. 3 threshold changed after a batch run (tables
    re-uploaded in place, same sizes) must reach the next batch run: each
    molecule's batch output equals its own single-context evaluation, and
    the changed one matches the oracle at its new cutoff."""
    import dataclasses

    from paper_2512_16677_gb300 import qmckl
    mols = cfg(4, walk_num=4)[:3]
    coords = [torch.from_numpy(m.coord).cuda() for m in mols]
    ctxs = _contexts(mols, coords)
    b = qmckl.Batch(ctxs)
    b.run()
    b.synchronize()
    ctxs[1].set_cutoff(1e-4)                          # T from 23.0 down to 9.2
    outs = b.run()
    b.synchronize()
    m1 = dataclasses.replace(mols[1], bits=None, eps=1e-4)
    _check_all(orc, [mols[0], m1, mols[2]], outs, n=32, seed=3)
    for c, m, o in zip(ctxs, mols, outs):
        single = c.mo_vgl_device()
        torch.cuda.synchronize()
        ref = single.double().cpu().numpy().reshape(-1, 5, m.mo_num)
        got = o.double().cpu().numpy().reshape(-1, 5, m.mo_num)
        assert np.max(np.abs(got - ref)) <= 1e-5 * np.abs(ref).max()


def test_batch_pairs_equal_single_sm(orc, cfg):
    """The batch's contraction on pairs of SMs (the default: M-tile pairs of
    each molecule, C blocked per molecule) and on single SMs multiply the
    same live blocks; the pair's extra k-steps add exact zeros.  Every
    molecule against the oracle and the two against each other."""
    from paper_2512_16677_gb300 import qmckl
    mols = cfg(4, walk_num=8)
    coords = [torch.from_numpy(m.coord).cuda() for m in mols]
    ctxs = _contexts(mols, coords)
    res = {}
    for pairs in (True, False):
        b = qmckl.Batch(ctxs)
        b.set_sm_pairs(pairs)
        outs = b.run()
        b.synchronize()
        res[pairs] = [o.double().cpu().numpy().reshape(-1, 5, m.mo_num) for o, m in zip(outs, mols)]
        if pairs:
            _check_all(orc, mols, outs, n=16, seed=4)
    for m, a, s in zip(mols, res[True], res[False]):
        assert np.max(np.abs(a - s)) <= 1e-6 * np.abs(s).max(), m.name


def test_batch_tf32_pairs(orc, cfg):
    """TF32 batch (pair contraction over FP32 blocked C): every molecule
    within the TF32 bar of the oracle and equal to its own context."""
    from paper_2512_16677_gb300 import qmckl
    mols = cfg(4, walk_num=4)[:5]
    ctxs = []
    for m in mols:
        ctx = qmckl.Context("tf32")
        ctx.set_molecule(m)
        ctx.set_points_device(torch.from_numpy(m.coord).cuda())
        ctxs.append(ctx)
    b = qmckl.Batch(ctxs)
    outs = b.run()
    b.synchronize()
    rng = np.random.default_rng(6)
    for c, m, o in zip(ctxs, mols, outs):
        got = o.double().cpu().numpy().reshape(-1, 5, m.mo_num)
        idx = np.sort(rng.choice(m.point_num, min(12, m.point_num), replace=False))
        ref, size = orc.mo_vgl(m, points=m.points[idx])
        assert_within("tf32", got[idx], ref, size, m.name)
        single = c.mo_vgl_device()
        torch.cuda.synchronize()
        s = single.double().cpu().numpy().reshape(-1, 5, m.mo_num)
        assert np.max(np.abs(got - s)) <= 1e-5 * np.abs(s).max(), m.name
