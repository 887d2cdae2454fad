"""Sampled parity at full size: which points to check, and the oracle on them.

The full workloads are too large for the FP64 oracle to evaluate whole, so
the GPU tests check a sample of points.  The sample is stratified over the
contraction's tiles (25 point slots each, cut from the spatial order of the
points) so that it reaches every kind of tile and every row position of a
tile:

* tiles ranked by their number of live (tile, AO chunk) blocks and split
  into equal strata, from the sparsest (points far from most nuclei) through
  mixed to the densest (points among many nuclei), the extremes included;
* the first and the last tile of the launch;
* slot offsets 0..24 inside the chosen tiles in rotation, so that every row
  group of a tile (5 rows per point) is written back through the permutation
  at least once;
* the first and last slot of the permutation and the first and last point in
  the caller's order.

The oracle is plain C called through ctypes, which releases the GIL, so a
thread pool over disjoint point ranges runs it on every host core.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

TILE = 25


def stratified_points(perm: np.ndarray, live: np.ndarray, n_points: int, seed: int = 0,
                      strata: int = 8) -> np.ndarray:
    """Caller point indices (sorted, unique) of about n_points sampled points;
    perm[s] = point at slot s, live[t] = live blocks of tile t."""
    rng = np.random.default_rng(seed)
    n = perm.shape[0]
    tiles = live.shape[0]
    per_tile = 8 if n_points >= 8 * strata else 1
    n_tiles = max(1, min(tiles, n_points // per_tile))
    order = np.argsort(live, kind="stable")            # sparsest tiles first
    chosen = [int(order[0]), int(order[-1]), 0, tiles - 1]
    bounds = np.linspace(0, tiles, strata + 1).astype(int)
    per_stratum = max(1, -(-(n_tiles - len(chosen)) // strata) + 1)
    for s in range(strata):
        lo, hi = bounds[s], bounds[s + 1]
        if hi <= lo:
            continue
        k = min(per_stratum, hi - lo)
        chosen.extend(int(t) for t in order[lo + rng.choice(hi - lo, k, replace=False)])
    seen = set()
    tiles_sel = [t for t in chosen if not (t in seen or seen.add(t))]
    slots = []
    for i, t in enumerate(tiles_sel):
        for j in range(per_tile):
            s = TILE * t + (i * per_tile + j) % TILE
            if s < n:
                slots.append(s)
    slots.extend([0, n - 1])
    pts = set(int(perm[s]) for s in slots)
    pts.update([0, n - 1])
    return np.array(sorted(pts), dtype=np.int64)


def slot_offsets_covered(perm: np.ndarray, idx: np.ndarray) -> set:
    """Slot offsets inside a tile (0..24) that the sampled points occupy."""
    where = np.empty_like(perm)
    where[perm] = np.arange(perm.shape[0], dtype=perm.dtype)
    return set(int(x) for x in where[idx] % TILE)


def mo_vgl_threaded(orc, mol, points: np.ndarray, threads: int | None = None):
    """orc.mo_vgl over disjoint ranges of points on a thread pool."""
    threads = threads or os.cpu_count() or 1
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 3)
    parts = [p for p in np.array_split(pts, max(1, min(threads, pts.shape[0]))) if p.shape[0]]
    with ThreadPoolExecutor(max_workers=len(parts)) as ex:
        res = list(ex.map(lambda p: orc.mo_vgl(mol, points=p), parts))
    return (np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res]))
