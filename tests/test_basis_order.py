"""The library's internal shell order (host logic, no GPU): bases listed
along a chain keep the caller's nucleus order, a basis in random atom order
is taken in Morton order of its nuclei, the mode switch forces either, and
the shells are split into a compact and a diffuse class by minimum
exponent (mode 1 keeps the caller's shell order untouched)."""
import numpy as np
import pytest

from paper_2512_16677_gb300 import synth


@pytest.fixture(scope="module")
def qk():
    from paper_2512_16677_gb300 import buildlib, qmckl
    buildlib.build()
    return qmckl


def _order(qk, m, mode=None):
    c = qk.Context("fp64")
    if mode is not None:
        c.set_basis_order(mode)
    c.set_molecule(m)
    return c.basis_order_spatial()


def test_chain_keeps_caller_order(qk):
    assert not _order(qk, synth.make_config(2, walk_num=1))
    assert not _order(qk, synth.make_config(3, walk_num=1))


def test_random_atom_order_goes_spatial(qk):
    assert _order(qk, synth.make_config(5, walk_num=1))


def relist_shells(m, nucleus_order):
    """The same molecule with its shells listed nucleus by nucleus in
    `nucleus_order` (primitives, AO factors and MO columns follow)."""
    l = m.shell_ang_mom
    nc = (l + 1) * (l + 2) // 2
    p0 = np.concatenate([[0], np.cumsum(m.shell_prim_num)])
    a0 = np.concatenate([[0], np.cumsum(nc)])
    rank = np.empty(m.nucl_num, dtype=np.int64)
    rank[np.asarray(nucleus_order)] = np.arange(m.nucl_num)
    sh = np.argsort(rank[m.shell_nucleus], kind="stable")
    prims = np.concatenate([np.arange(p0[s], p0[s + 1]) for s in sh])
    aos = np.concatenate([np.arange(a0[s], a0[s + 1]) for s in sh])
    return synth.Molecule(**{**m.__dict__,
                             "shell_nucleus": m.shell_nucleus[sh], "shell_ang_mom": l[sh],
                             "shell_prim_num": m.shell_prim_num[sh],
                             "shell_factor": m.shell_factor[sh],
                             "exponent": m.exponent[prims], "coefficient": m.coefficient[prims],
                             "prim_factor": m.prim_factor[prims],
                             "ao_factor": m.ao_factor[aos],
                             "mo_coef": np.ascontiguousarray(m.mo_coef[:, aos])}), aos


def test_shuffled_chain_goes_spatial(qk):
    m = synth.make_config(3, walk_num=1)
    m2, _ = relist_shells(m, np.random.default_rng(5).permutation(m.nucl_num))
    assert _order(qk, m2)


def test_mode_switch(qk):
    m = synth.make_config(1, walk_num=1)
    assert not _order(qk, m, 1)
    assert not _order(qk, synth.make_config(5, walk_num=1), 1)
    assert _order(qk, synth.make_config(3, walk_num=1), 2)
    c = qk.Context("fp64")
    with pytest.raises(qk.QmcklError) as e:
        c.set_basis_order(3)
    assert e.value.status == -1


def _classes(m):
    """compact[s]: minimum exponent of caller shell s >= that of the shell
    holding the AO-weighted median, shells ranked by descending minimum."""
    p0 = np.concatenate([[0], np.cumsum(m.shell_prim_num)])
    gmin = np.array([m.exponent[p0[s]:p0[s + 1]].min() for s in range(m.shell_num)])
    nc = (m.shell_ang_mom + 1) * (m.shell_ang_mom + 2) // 2
    by = np.argsort(-gmin, kind="stable")
    cum = np.cumsum(nc[by])
    gmed = gmin[by[np.argmax(2 * cum >= m.ao_num)]]
    return gmin >= gmed


def _shell_order(qk, m, mode=None):
    c = qk.Context("fp64")
    if mode is not None:
        c.set_basis_order(mode)
    c.set_molecule(m)
    return c.shell_order(m.shell_num)


@pytest.mark.parametrize("cfg_i", [2, 3, 5, 6])
def test_compact_then_diffuse(qk, cfg_i):
    m = synth.make_config(cfg_i, walk_num=1)
    order = _shell_order(qk, m)
    np.testing.assert_array_equal(np.sort(order), np.arange(m.shell_num))
    compact = _classes(m)
    k = int(compact.sum())
    assert 0 < k < m.shell_num
    assert compact[order[:k]].all() and not compact[order[k:]].any()
    if cfg_i in (2, 3):  # chains: each class keeps the caller's order
        assert np.all(np.diff(order[:k]) > 0) and np.all(np.diff(order[k:]) > 0)
    else:                # Morton nuclei: a nucleus's shells of a class stay together
        for part in (order[:k], order[k:]):
            nuc = m.shell_nucleus[part]
            starts = nuc[np.r_[True, nuc[1:] != nuc[:-1]]]
            assert len(starts) == len(np.unique(nuc))


def test_caller_mode_is_identity(qk):
    m = synth.make_config(5, walk_num=1)
    np.testing.assert_array_equal(_shell_order(qk, m, 1), np.arange(m.shell_num))
    c = qk.Context("fp64")
    with pytest.raises(qk.QmcklError) as e:
        c.shell_order(1)
    assert e.value.status == -4
