"""Multi-rank walker sharding on the CPU (gloo, world size 2).

Each rank takes its contiguous walker range, computes dL/dC and dL/dR_nuc of
its shard (the oracle stands in for the device work, which needs a GPU), and
the gradients are summed with the library's all-reduce helper.  The sum must
equal the unsharded gradient to rounding.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2512_16677_gb300 import parallel, synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle
    m = synth.make_config(1)
    W = synth.random_weights(np.random.default_rng(30), m.point_num, m.mo_num)
    W = W.reshape(m.walk_num, m.elec_num, 5, m.mo_num)
    b, e = parallel.shard_range(m.walk_num, rank, world)
    shard = m.with_points(m.coord[b:e])
    dC, dR = oracle.adjoint(shard, W[b:e].reshape(-1, 5, m.mo_num))
    tC, tR = torch.from_numpy(dC), torch.from_numpy(dR)
    parallel.allreduce_gradients(tC, tR)
    if rank == 0:
        np.savez(out_path, dC=tC.numpy(), dR=tR.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_adjoint_allreduce(tmp_path, orc):
    world = 2
    out = str(tmp_path / "g.npz")
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    m = synth.make_config(1)
    W = synth.random_weights(np.random.default_rng(30), m.point_num, m.mo_num)
    dC, dR, dCs, dRs = orc.adjoint(m, W, sizes=True)
    g = np.load(out)
    assert np.max(np.abs(g["dC"] - dC) / dCs) < 1e-14
    assert np.max(np.abs(g["dR"] - dR) / dRs) < 1e-14


def test_shard_ranges_partition():
    for n in (1, 7, 64, 256):
        for world in (1, 2, 3, 8):
            rs = [parallel.shard_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        parallel.shard_range(4, 2, 2)
