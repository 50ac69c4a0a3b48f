"""The sharded (multi-rank) path on CPU: 2 gloo ranks, each running the FP64
oracle on its contiguous shard; forward results and the all-reduced training
gradients must equal the unsharded computation."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2304_12745_gb300 import channels as ch
from paper_2304_12745_gb300.sharding import allreduce_mean, shard_range

B, K, M, T = 37, 4, 16, 5


def _inputs():
    H = ch.rayleigh(B, K, M, seed=123).astype(np.complex128)
    t = np.ones((B, K))
    mu = ch.uniform_steps(T, 0.02, 0.08, seed=124).astype(np.float64)
    return H, t, mu


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    H, t, mu = _inputs()
    lo, hi = shard_range(B, rank, world)
    W, obj, res, st = oracle.batch_forward(1, H[lo:hi], t[lo:hi], mu)
    grads = [oracle.ufproj_grad(H[b], t[b], mu, 1.0) for b in range(lo, hi)]
    loss_l = torch.tensor([np.mean([g[0] for g in grads])])
    dmu_l = torch.tensor(np.mean([g[1] for g in grads], axis=0))
    loss, dmu, _ = allreduce_mean(loss_l, dmu_l, None, hi - lo)
    # forward results: gather every shard's objectives on every rank
    obj_t = torch.zeros(B, dtype=torch.float64)
    obj_t[lo:hi] = torch.from_numpy(obj)
    dist.all_reduce(obj_t)
    out[rank] = (loss.item(), dmu.numpy().copy(), obj_t.numpy().copy())
    dist.destroy_process_group()


def test_shard_ranges_cover_batch_exactly():
    for Bn in (1, 7, 64, 65537):
        for world in (1, 2, 3, 8):
            rs = [shard_range(Bn, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == Bn
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            sizes = [hi - lo for lo, hi in rs]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def test_two_gloo_ranks_match_unsharded(orc):
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    H, t, mu = _inputs()
    W, obj, _, _ = orc.batch_forward(1, H, t, mu)
    grads = [orc.ufproj_grad(H[b], t[b], mu, 1.0) for b in range(B)]
    loss_ref = np.mean([g[0] for g in grads])
    dmu_ref = np.mean([g[1] for g in grads], axis=0)
    for r in range(world):
        loss, dmu, obj_all = res[r]
        assert loss == pytest.approx(loss_ref, rel=1e-12)
        assert np.allclose(dmu, dmu_ref, rtol=1e-12, atol=1e-14)
        assert np.array_equal(obj_all, obj)
