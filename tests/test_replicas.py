"""Data-parallel replicas on CPU: two gloo ranks.

Each rank takes its shard of one basket, computes the per-track adjoint of its
tracks with the oracle (the CPU stand-in for the kernel), sums its geometry
gradients per owner, and the ranks combine them with allreduce_geometry.  The
result must equal the single-process sum over the whole basket, be the same
bits on both ranks, and the timing / shard helpers must behave as documented.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1312_0816_gb300 import replicas, scenes  # noqa: E402

N = 3001   # odd: the shards differ in size


def owner_sums(sc, adj, a, b):
    nd = sc.n_daughters
    gt = np.zeros((max(nd, 1), 3))
    gp = np.zeros((nd + 1, 5))
    for i in range(a, b):
        if not adj["ok"][i]:
            continue
        j = int(adj["winner"][i])
        o = nd if j < 0 else j
        if j >= 0:
            gt[j] += adj["gt"][:, i]
        gp[o] += adj["gparams"][:, i]
    return gt[:nd], gp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import oracle

    try:
        assert replicas.init("gloo")
        assert replicas.env() == (world, rank, rank)
        sc = scenes.diff3()
        tr = scenes.sample_tracks(sc, N, 7)
        off, cnt = replicas.shard(N, world, rank)
        part = tr.slice(off, off + cnt)
        adj = oracle.adjoint(sc, part)
        gt, gp = owner_sums(sc, adj, 0, cnt)
        tgt, tgp = torch.from_numpy(gt.copy()), torch.from_numpy(gp.copy())
        replicas.allreduce_geometry(tgt, tgp, None)
        mx = replicas.max_over_ranks(float(rank + 1))
        tot = replicas.sum_over_ranks(float(cnt))
        replicas.barrier()
        out[rank] = (tgt.numpy().copy(), tgp.numpy().copy(), mx, tot, off, cnt)
    finally:
        if tdist.is_initialized():
            tdist.destroy_process_group()


def test_shard_partitions_exactly():
    for n in (0, 1, 7, 1024, 3001):
        for world in (1, 2, 3, 8):
            spans = [replicas.shard(n, world, r) for r in range(world)]
            assert spans[0][0] == 0
            for (o0, c0), (o1, _) in zip(spans, spans[1:]):
                assert o0 + c0 == o1
            assert sum(c for _, c in spans) == n
            assert max(c for _, c in spans) - min(c for _, c in spans) <= 1
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)


def test_single_process_helpers_are_identity():
    assert not replicas.active()
    assert replicas.max_over_ranks(3.5) == 3.5
    t = torch.ones(3, dtype=torch.float64)
    replicas.allreduce_geometry(t)
    assert torch.equal(t, torch.ones(3, dtype=torch.float64))


def test_two_gloo_ranks_sum_geometry_gradients(orc):
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    sc = scenes.diff3()
    tr = scenes.sample_tracks(sc, N, 7)
    adj = orc.adjoint(sc, tr)
    gt_full, gp_full = owner_sums(sc, adj, 0, N)
    for r in range(world):
        gt, gp, mx, tot, off, cnt = res[r]
        assert mx == float(world)
        assert tot == float(N)
        assert np.allclose(gt, gt_full, rtol=1e-12, atol=1e-12)
        assert np.allclose(gp, gp_full, rtol=1e-12, atol=1e-12)
        # both ranks hold the same bits
        assert np.array_equal(gt, res[0][0]) and np.array_equal(gp, res[0][1])
    assert res[0][4] == 0 and res[1][4] == res[0][5]
