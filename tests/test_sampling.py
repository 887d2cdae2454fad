"""Host logic of the full-size parity sample (tests/sampling.py)."""
import numpy as np

from sampling import TILE, mo_vgl_threaded, slot_offsets_covered, stratified_points


def test_stratified_sample_reaches_every_tile_class_and_slot():
    rng = np.random.default_rng(3)
    n = 153600
    perm = rng.permutation(n).astype(np.int32)
    live = rng.integers(0, 29, size=n // TILE).astype(np.int32)
    live[17] = -1          # a unique sparsest tile
    live[4000] = 99        # a unique densest tile
    idx = stratified_points(perm, live, 1024, seed=7)
    assert idx.shape[0] >= 1024
    assert np.all(np.diff(idx) > 0)
    assert slot_offsets_covered(perm, idx) == set(range(TILE))
    where = np.empty_like(perm)
    where[perm] = np.arange(n, dtype=np.int32)
    tiles = set((where[idx] // TILE).tolist())
    assert {17, 4000, 0, n // TILE - 1} <= tiles
    assert {0, n - 1, int(perm[0]), int(perm[-1])} <= set(idx.tolist())
    # every stratum of the live-block ranking is represented
    rank = np.empty(n // TILE, dtype=np.int64)
    rank[np.argsort(live, kind="stable")] = np.arange(n // TILE)
    strata = set((rank[sorted(tiles)] * 8 // (n // TILE)).tolist())
    assert strata == set(range(8))


def test_threaded_oracle_equals_single_call(orc, cfg):
    m = cfg(1)
    pts = m.points[:37]
    a, sa = orc.mo_vgl(m, points=pts)
    b, sb = mo_vgl_threaded(orc, m, pts, threads=4)
    assert np.array_equal(a, b) and np.array_equal(sa, sb)
