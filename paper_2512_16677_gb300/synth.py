"""Seeded synthetic inputs shaped like the paper's orbital workloads.

This module only *draws* inputs: nuclear geometries, Gaussian basis sets
(exponents, contraction coefficients and the normalisation constants that a
basis-set file carries alongside them), MO coefficients and electron
positions.  It evaluates no orbital, performs no screening and no
contraction; both the CUDA library and the CPU oracle receive what it draws.

Conventions (all lengths in bohr, exponents in bohr^-2):

* Shells follow Eq. 2 with Gaussian primitives (p = 2) and n_s = 0.
* The per-primitive factor f_ks normalises the x^l Cartesian component of a
  primitive, the shell factor N_s normalises the contracted x^l component,
  and the per-AO factor M_n of Eq. 1 rescales every other Cartesian
  component (a, b, c) of the shell to unit norm (the GAMESS convention the
  paper mentions in Sec. 3.1).
* Cartesian components inside a shell are ordered lexicographically by
  descending (a, b): l=2 -> xx, xy, xz, yy, yz, zz.
* Points are laid out [walk][elec][3]; point index p = walk * elec_num + elec.

Five workloads are provided (``make_config(1..5)``); see ``CONFIGS``.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

ANGSTROM = 1.8897261246  # bohr per angstrom
SEED_BASE = 2512166770
ELEMENT_Z = {"H": 1, "C": 6, "N": 7, "O": 8, "Cu": 29}


def cartesian_powers(l: int) -> List[Tuple[int, int, int]]:
    """(a, b, c) triples of a Cartesian shell, descending lexicographic."""
    out = []
    for a in range(l, -1, -1):
        for b in range(l - a, -1, -1):
            out.append((a, b, l - a - b))
    return out


def _dfact(n: int) -> float:
    """Double factorial with (-1)!! = 0!! = 1."""
    r = 1.0
    while n > 1:
        r *= n
        n -= 2
    return r


@dataclasses.dataclass
class Molecule:
    """One system: nuclei, basis, MO coefficients, points and cutoff."""

    name: str
    nucl_charge: np.ndarray      # [nucl] float64
    nucl_coord: np.ndarray       # [nucl][3] float64, bohr
    shell_nucleus: np.ndarray    # [shell] int64
    shell_ang_mom: np.ndarray    # [shell] int32
    shell_prim_num: np.ndarray   # [shell] int64
    shell_factor: np.ndarray     # [shell] float64  (N_s)
    exponent: np.ndarray         # [prim] float64   (gamma_ks), shell-major
    coefficient: np.ndarray      # [prim] float64   (a_ks)
    prim_factor: np.ndarray      # [prim] float64   (f_ks)
    ao_factor: np.ndarray        # [ao] float64     (M_n)
    mo_coef: np.ndarray          # [mo][ao] float64 (C_nk)
    coord: np.ndarray            # [walk][elec][3] float64, bohr
    bits: Optional[int] = 53     # precision parameter B of Eq. 3
    eps: Optional[float] = None  # alternative: cutoff on exp(-gamma r^2)

    @property
    def nucl_num(self) -> int:
        return int(self.nucl_charge.shape[0])

    @property
    def shell_num(self) -> int:
        return int(self.shell_ang_mom.shape[0])

    @property
    def prim_num(self) -> int:
        return int(self.exponent.shape[0])

    @property
    def ao_num(self) -> int:
        return int(self.ao_factor.shape[0])

    @property
    def mo_num(self) -> int:
        return int(self.mo_coef.shape[0])

    @property
    def walk_num(self) -> int:
        return int(self.coord.shape[0])

    @property
    def elec_num(self) -> int:
        return int(self.coord.shape[1])

    @property
    def point_num(self) -> int:
        return self.walk_num * self.elec_num

    @property
    def points(self) -> np.ndarray:
        """Points as a contiguous [point][3] float64 array."""
        return np.ascontiguousarray(self.coord.reshape(-1, 3))

    def with_points(self, coord: np.ndarray) -> "Molecule":
        """Same system, other points ([walk][elec][3] or [n][3])."""
        c = np.asarray(coord, dtype=np.float64)
        if c.ndim == 2:
            c = c.reshape(1, c.shape[0], 3)
        return dataclasses.replace(self, coord=np.ascontiguousarray(c))

    def with_walkers(self, walk_num: int) -> "Molecule":
        """Keep the first walk_num walkers."""
        return dataclasses.replace(
            self, coord=np.ascontiguousarray(self.coord[:walk_num]))


# ---------------------------------------------------------------------------
# basis recipes
# ---------------------------------------------------------------------------

# (l, nprim range, exponent range) per shell of an element's basis
_Recipe = List[Tuple[int, Tuple[int, int], Tuple[float, float]]]

_GEN_S = (1, 8), (0.1, 5000.0)   # generic shell rule: nprim U{1..8}, gamma logU
RECIPE_SMALL: Dict[str, _Recipe] = {
    # O/C/N 3s2p1d, H 2s1p; every shell drawn with the generic rule
    "O": [(0, *_GEN_S)] * 3 + [(1, *_GEN_S)] * 2 + [(2, *_GEN_S)],
    "C": [(0, *_GEN_S)] * 3 + [(1, *_GEN_S)] * 2 + [(2, *_GEN_S)],
    "N": [(0, *_GEN_S)] * 3 + [(1, *_GEN_S)] * 2 + [(2, *_GEN_S)],
    "H": [(0, *_GEN_S)] * 2 + [(1, *_GEN_S)],
    "Cu": [(0, *_GEN_S)] * 4 + [(1, *_GEN_S)] * 3 + [(2, *_GEN_S)] * 2,
}
_S = (0, (1, 8), (0.1, 5000.0))
_P = (1, (1, 4), (0.1, 500.0))
_D = (2, (1, 1), (0.1, 5.0))
_F = (3, (1, 1), (0.1, 5.0))
RECIPE_TZ: Dict[str, _Recipe] = {
    # heavy atoms [2s1p1d1f] (21 Cartesian AOs), H [1s]
    "C": [_S, _S, _P, _D, _F],
    "N": [_S, _S, _P, _D, _F],
    "O": [_S, _S, _P, _D, _F],
    "H": [_S],
}


def _norm_prim(gamma: np.ndarray, l: int) -> np.ndarray:
    """f_ks: unit norm of a primitive's x^l component."""
    return ((2.0 * gamma / math.pi) ** 0.75 * (4.0 * gamma) ** (0.5 * l)
            / math.sqrt(_dfact(2 * l - 1)))


def _norm_shell(gamma: np.ndarray, a: np.ndarray, f: np.ndarray, l: int) -> float:
    """N_s: unit norm of the contracted x^l component."""
    gi = gamma[:, None] + gamma[None, :]
    ov = (math.pi / gi) ** 1.5 * _dfact(2 * l - 1) / (2.0 * gi) ** l
    s = float(np.sum((a * f)[:, None] * (a * f)[None, :] * ov))
    return 1.0 / math.sqrt(s)


def _norm_ao(l: int) -> List[float]:
    """M_n for each Cartesian (a,b,c): rescales to unit norm."""
    return [math.sqrt(_dfact(2 * l - 1)
                      / (_dfact(2 * a - 1) * _dfact(2 * b - 1) * _dfact(2 * c - 1)))
            for (a, b, c) in cartesian_powers(l)]


def build_basis(rng: np.random.Generator, elements: Sequence[str],
                recipe: Dict[str, _Recipe]):
    """Draw one shell set per nucleus from its element's recipe."""
    sh_nuc, sh_l, sh_np, sh_fac = [], [], [], []
    expo, coef, pfac, aofac = [], [], [], []
    for ia, el in enumerate(elements):
        for (l, (nlo, nhi), (glo, ghi)) in recipe[el]:
            n = int(rng.integers(nlo, nhi + 1))
            g = np.exp(rng.uniform(math.log(glo), math.log(ghi), size=n))
            a = rng.uniform(0.1, 1.0, size=n)
            f = _norm_prim(g, l)
            sh_nuc.append(ia)
            sh_l.append(l)
            sh_np.append(n)
            sh_fac.append(_norm_shell(g, a, f, l))
            expo.extend(g.tolist())
            coef.extend(a.tolist())
            pfac.extend(f.tolist())
            aofac.extend(_norm_ao(l))
    return (np.array(sh_nuc, dtype=np.int64), np.array(sh_l, dtype=np.int32),
            np.array(sh_np, dtype=np.int64), np.array(sh_fac),
            np.array(expo), np.array(coef), np.array(pfac), np.array(aofac))


# ---------------------------------------------------------------------------
# geometries and electrons
# ---------------------------------------------------------------------------

def _unit_vectors(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def self_avoiding_chain(rng, n: int, bond=(1.1, 1.5), min_dist=1.0,
                        tries=2000) -> np.ndarray:
    """3D random chain (angstrom); non-bonded atoms keep min_dist apart."""
    pos = np.zeros((n, 3))
    for i in range(1, n):
        for _ in range(tries):
            cand = pos[i - 1] + rng.uniform(*bond) * _unit_vectors(rng, 1)[0]
            if i < 2 or np.min(np.linalg.norm(pos[: i - 1] - cand, axis=1)) >= min_dist:
                pos[i] = cand
                break
        else:
            raise RuntimeError("self-avoiding chain: no free position")
    return pos - pos.mean(axis=0)


def packed_cluster(rng, n: int, radius: float, min_dist=1.0,
                   tries=100000) -> np.ndarray:
    """Random sequential addition of n points in a sphere (angstrom)."""
    pos = np.zeros((0, 3))
    for _ in range(n):
        for _ in range(tries):
            c = rng.uniform(-radius, radius, size=3)
            if c @ c > radius * radius:
                continue
            if pos.shape[0] == 0 or np.min(np.sum((pos - c) ** 2, axis=1)) >= min_dist ** 2:
                pos = np.vstack([pos, c])
                break
        else:
            raise RuntimeError("packed cluster: no free position")
    return pos


def assign_electrons(charges: np.ndarray, elec_num: int) -> np.ndarray:
    """Electron count per nucleus proportional to Z (largest remainder)."""
    q = elec_num * charges / charges.sum()
    base = np.floor(q).astype(np.int64)
    rem = elec_num - int(base.sum())
    order = np.argsort(-(q - base), kind="stable")
    base[order[:rem]] += 1
    return base


def place_electrons(rng, nucl_coord_bohr: np.ndarray, counts: np.ndarray,
                    walk_num: int, sigma_ang=0.7) -> np.ndarray:
    """[walk][elec][3] Gaussian clouds around the nuclei (bohr)."""
    centres = np.repeat(nucl_coord_bohr, counts, axis=0)
    sig = sigma_ang * ANGSTROM
    return centres[None, :, :] + sig * rng.normal(size=(walk_num, centres.shape[0], 3))


def element_counts(ratio: Dict[str, int], n: int) -> List[str]:
    """Split n nuclei over elements in the given ratio (largest remainder)."""
    names = list(ratio)
    w = np.array([ratio[k] for k in names], dtype=np.float64)
    q = n * w / w.sum()
    base = np.floor(q).astype(np.int64)
    order = np.argsort(-(q - base), kind="stable")
    base[order[: n - int(base.sum())]] += 1
    out: List[str] = []
    for k, c in zip(names, base):
        out += [k] * int(c)
    return out


def make_molecule(name, rng, elements, pos_ang, recipe, mo_num, elec_num,
                  walk_num, bits=None, eps=None) -> Molecule:
    charges = np.array([ELEMENT_Z[e] for e in elements], dtype=np.float64)
    coord_n = np.ascontiguousarray(pos_ang * ANGSTROM)
    basis = build_basis(rng, elements, recipe)
    ao_num = basis[-1].shape[0]
    C = rng.normal(size=(mo_num, ao_num)) / math.sqrt(ao_num)
    counts = assign_electrons(charges, elec_num)
    pts = place_electrons(rng, coord_n, counts, walk_num)
    return Molecule(name, charges, coord_n, *basis, C, np.ascontiguousarray(pts),
                    bits=bits, eps=eps)


# ---------------------------------------------------------------------------
# the five workloads
# ---------------------------------------------------------------------------

CONFIGS = {
    1: "water: 3 nuclei, O 3s2p1d + H 2s1p (25 Cartesian AOs), 5 MOs, "
       "10 e- x 64 walkers, B = 53",
    2: "organic chain: 150 nuclei C:N:O:H 56:10:9:75, heavy [2s1p1d1f] H [1s] "
       "(1650 AOs), 300 MOs, 600 e- x 256 walkers, eps = 1e-10",
    3: "adjoint chain: 50 nuclei C/H alternating, C 3s2p1d H 2s1p (500 AOs), "
       "100 MOs, 200 e- x 128 walkers, B = 53",
    4: "uneven batch: 12 chains of 20-200 nuclei, organic mix and basis, "
       "4 e-/nucleus, 16-256 walkers, MOs = e-/2, eps = 1e-10",
    5: "large cluster: 1000 nuclei C:O:H 400:100:500 in 10^4 A^3, C/O 3s2p1d "
       "H 2s1p (10000 AOs), 2000 MOs, 4000 e- x 16 walkers, eps = 1e-10",
    6: "density stand-in: 104 nuclei C:N:O:H:Cu 34:11:10:48:1 in a sphere of 1040 A^3, "
       "C/N/O 3s2p1d, H 2s1p, Cu 4s3p2d (1090 AOs), 218 doubly occupied MOs, "
       "100^3 grid over the nuclei +- 4 bohr, eps = 1e-10",
}


def make_config(idx: int, walk_num: Optional[int] = None):
    """Draw workload ``idx`` (1..6).  Config 4 returns a list of molecules.

    ``walk_num`` overrides the walker count (used for reduced test sizes);
    every other draw is unchanged, so the first walkers match the full case.
    """
    rng = np.random.default_rng(np.random.PCG64(SEED_BASE + idx))
    if idx == 1:
        el = ["O", "H", "H"]
        pos = np.array([[0.0, 0.0, 0.0], [0.76, 0.0, 0.59], [-0.76, 0.0, 0.59]])
        m = make_molecule("water", rng, el, pos, RECIPE_SMALL, 5, 10, 64, bits=53)
    elif idx == 2:
        el = element_counts({"C": 56, "N": 10, "O": 9, "H": 75}, 150)
        el = [el[i] for i in rng.permutation(len(el))]
        pos = self_avoiding_chain(rng, 150)
        m = make_molecule("organic150", rng, el, pos, RECIPE_TZ, 300, 600, 256, eps=1e-10)
    elif idx == 3:
        el = ["C", "H"] * 25
        pos = self_avoiding_chain(rng, 50)
        m = make_molecule("chain50", rng, el, pos, RECIPE_SMALL, 100, 200, 128, bits=53)
    elif idx == 4:
        mols = []
        for i in range(12):
            n = int(round(math.exp(rng.uniform(math.log(20), math.log(200)))))
            w = int(round(math.exp(rng.uniform(math.log(16), math.log(256)))))
            el = element_counts({"C": 56, "N": 10, "O": 9, "H": 75}, n)
            el = [el[j] for j in rng.permutation(len(el))]
            pos = self_avoiding_chain(rng, n)
            ne = 4 * n
            mols.append(make_molecule(f"batch{i}_{n}", rng, el, pos, RECIPE_TZ,
                                      ne // 2, ne, w, eps=1e-10))
        if walk_num is not None:
            mols = [mm.with_walkers(min(walk_num, mm.walk_num)) for mm in mols]
        return mols
    elif idx == 6:
        # stand-in for the density workload of Sec. 5.4 (a Cu(II)-peptide
        # complex in a double-zeta basis: ~1100 AOs, 218 occupied MOs)
        el = element_counts({"C": 34, "N": 11, "O": 10, "H": 48, "Cu": 1}, 104)
        el = [el[i] for i in rng.permutation(len(el))]
        radius = (3.0 * 10.0 * 104 / (4.0 * math.pi)) ** (1.0 / 3.0)
        pos = packed_cluster(rng, 104, radius)
        m = make_molecule("peptide104", rng, el, pos, RECIPE_SMALL, 218, 436, 1, eps=1e-10)
    elif idx == 5:
        el = element_counts({"C": 400, "O": 100, "H": 500}, 1000)
        el = [el[i] for i in rng.permutation(len(el))]
        radius = (3.0 * 10000.0 / (4.0 * math.pi)) ** (1.0 / 3.0)
        pos = packed_cluster(rng, 1000, radius)
        m = make_molecule("cluster1000", rng, el, pos, RECIPE_SMALL, 2000, 4000, 16,
                          eps=1e-10)
    else:
        raise ValueError(f"unknown config {idx}")
    if walk_num is not None:
        m = m.with_walkers(walk_num)
    return m


def density_grid(mol: Molecule, n: int = 100, margin: float = 4.0):
    """(origin, spacing, counts) of an n^3 grid over the nuclei's bounding
    box widened by ``margin`` bohr on every side (Sec. 5.4's 100^3 grid)."""
    lo = mol.nucl_coord.min(axis=0) - margin
    hi = mol.nucl_coord.max(axis=0) + margin
    return lo, (hi - lo) / (n - 1), (n, n, n)


def occupations(mol: Molecule) -> np.ndarray:
    """Occupation weights of the density workloads: 2 for every MO."""
    return np.full(mol.mo_coef.shape[0], 2.0)


def cusp_radii(mol: Molecule) -> np.ndarray:
    """Cusp-correction radii for tests and measurement: 0.5 / sqrt(Z) bohr
    per nucleus (0.5 for H, 0.20 for C, 0.18 for O)."""
    return 0.5 / np.sqrt(np.asarray(mol.nucl_charge, dtype=np.float64))


def random_weights(rng: np.random.Generator, point_num: int, mo_num: int) -> np.ndarray:
    """Loss weights W [point][5][mo] for the adjoint workload, U(-1, 1)."""
    return rng.uniform(-1.0, 1.0, size=(point_num, 5, mo_num))


def tiny_shell(l: int, gammas: Sequence[float], coefs: Sequence[float],
               centre=(0.0, 0.0, 0.0), points: Optional[np.ndarray] = None,
               mo_coef: Optional[np.ndarray] = None, bits=53) -> Molecule:
    """One nucleus carrying one shell: for closed-form and quadrature checks."""
    g = np.asarray(gammas, dtype=np.float64)
    a = np.asarray(coefs, dtype=np.float64)
    f = _norm_prim(g, l)
    ns = _norm_shell(g, a, f, l)
    ao = np.array(_norm_ao(l))
    pts = np.zeros((1, 1, 3)) if points is None else np.asarray(points).reshape(1, -1, 3)
    C = np.eye(ao.shape[0]) if mo_coef is None else mo_coef
    return Molecule("tiny", np.array([1.0]), np.array([centre], dtype=np.float64),
                    np.array([0], dtype=np.int64), np.array([l], dtype=np.int32),
                    np.array([g.shape[0]], dtype=np.int64), np.array([ns]),
                    g, a, f, ao, np.ascontiguousarray(C, dtype=np.float64),
                    np.ascontiguousarray(pts), bits=bits)
