"""The library's internal shell order (host logic, no GPU): bases listed
along a chain keep the caller's order, a basis in random atom order is
taken in Morton order of its nuclei, and the mode switch forces either."""
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
