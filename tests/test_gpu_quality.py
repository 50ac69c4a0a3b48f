"""The pieces of the paper-setting quality reproduction (Sec. VI) against the oracle.

* Per-layer PCG (Sec. VI-B) of the GPU's outputs after each of the 20 layers equals
  the FP64 oracle's, channel by channel, for PGD with the paper's parameters and for
  the projected layer, on test channels of the paper setting.
* The supervised labels: 4,000 projected layers with diminishing shrink on the GPU
  land within 0.3 % of the objective of the oracle's ADMM optimum of Eq. (optim1),
  and are feasible.
* The benchmark's sum-rate evaluation equals the oracle's O5 sum rate.
"""
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_12745_gb300 import channels as ch

pytestmark = pytest.mark.gpu

K, M = 8, 64
AMP = math.sqrt(10.0)


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12745_gb300 import capi, precoder
    return capi, precoder


def _test_channels(n):
    return ch.paper_set("test")[:n]


@pytest.mark.parametrize("layer", ["pgd", "proj"])
def test_per_layer_pcg_matches_oracle(pc, orc, layer):
    capi, precoder = pc
    B, T = 48, 20
    H = _test_channels(B)
    t = np.full((B, K), AMP)
    tK = torch.full((K,), AMP, device="cuda")
    Hd = torch.from_numpy(H).cuda()
    if layer == "pgd":
        mode = capi.LAYER_PGD
        step = np.full(T, ch.paper_eta(K, M), np.float32)
        lam = np.full(T, 1 / 15, np.float32)
    else:
        mode = capi.LAYER_PROJ
        step = np.linspace(0.3, 0.05, T).astype(np.float32)
        lam = None
    # oracle: every layer's output from one traced run per channel
    pcg_o = np.zeros((T, B))
    for b in range(B):
        Hb = H[b].astype(np.complex128)
        if layer == "pgd":
            _, tr = orc.ufpgd_forward(Hb, t[b], step.astype(np.float64), lam.astype(np.float64),
                                      trace=True)
        else:
            _, _, tr = orc.ufproj_forward(Hb, t[b], step.astype(np.float64), trace=True)
        for l in range(T):
            pcg_o[l, b] = orc.pcg(Hb, t[b], tr[l + 1])
    pz = precoder.Plan(capi.LAYER_PROJ, 1, [(M, K)], B, tensor_cores=True)
    obj_zf = pz.solve(Hd, tK, torch.zeros(1, device="cuda"))[1]
    pz.close()
    for TT in range(1, T + 1):
        pl = precoder.Plan(mode, TT, [(M, K)], B, tensor_cores=True)
        obj = pl.solve(Hd, tK, torch.from_numpy(step[:TT].copy()).cuda(),
                       None if lam is None else torch.from_numpy(lam[:TT].copy()).cuda())[1]
        pl.close()
        pcg_g = (obj_zf / obj).cpu().numpy()
        # a ratio of two objectives, each within 1e-5 of the oracle's
        assert np.max(np.abs(pcg_g / pcg_o[TT - 1] - 1)) <= 2e-5, TT


def test_long_run_labels_near_the_admm_optimum(pc, orc):
    capi, precoder = pc
    B, T = 32, 4000
    H = _test_channels(B)
    t = np.full((B, K), AMP)
    Wa, _, st = orc.batch_admm(H.astype(np.complex128), t, tol=1e-10, nthreads=8)
    assert np.all(st == orc.OK)
    oa = np.array([orc.l21(w) for w in Wa])
    mu = (0.1 / torch.sqrt(torch.arange(1, T + 1, device="cuda", dtype=torch.float32))).contiguous()
    pl = precoder.Plan(capi.LAYER_PROJ, T, [(M, K)], B, tensor_cores=True)
    W, obj, res, fl = pl.solve(torch.from_numpy(H).cuda(), torch.full((K,), AMP, device="cuda"), mu)
    torch.cuda.synchronize()
    pl.close()
    obj = obj.cpu().numpy()
    assert np.all(fl.cpu().numpy() == 0)
    gap = (obj - oa) / oa
    assert np.all(gap >= -1e-5) and gap.max() <= 3e-3, gap
    assert np.all(res.cpu().numpy() <= 1e-4 * AMP * math.sqrt(K))


def test_bench_sum_rate_matches_oracle(pc, orc):
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    B = 16
    H = _test_channels(B)
    rs = np.random.default_rng(3)
    W = (rs.standard_normal((B, K, M)) + 1j * rs.standard_normal((B, K, M))).astype(np.complex64) * 0.1
    r = bench.sum_rate_per_channel(torch, torch.from_numpy(H).cuda(), torch.from_numpy(W).cuda())
    r = r.cpu().numpy()
    ro = np.array([orc.sum_rate(H[b].astype(np.complex128), W[b].astype(np.complex128), 1.0)
                   for b in range(B)])
    assert np.allclose(r, ro, rtol=1e-5), (r, ro)
