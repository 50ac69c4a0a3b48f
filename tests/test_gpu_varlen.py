"""Uneven batches (bucketed, optionally one CUDA graph) on the GPU.

The workload follows the uneven benchmark: (M, K) drawn uniformly from
{(32,4), (64,8), (128,16), (256,32)}, Rician ULA channels (K-factor 0-10 dB),
unit targets, T = 10 projected layers.  Every instance must be bitwise equal to
the uniform solve of its shape (same kernel variant) and match the FP64 oracle
within the parity tolerances; rejected descriptors are flagged.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_12745_gb300 import channels as ch

pytestmark = pytest.mark.gpu


def pack(shapes, seed):
    """Concatenate per-instance Rician channels into one flat buffer + descriptors."""
    Hs, h_off, t_off, off, toff = [], [], [], 0, 0
    for b, (M, K) in enumerate(shapes):
        H = ch.rician_ula(1, int(K), int(M), seed=seed * 100003 + b)[0]
        Hs.append(H.reshape(-1))
        h_off.append(off)
        t_off.append(toff)
        off += H.size
        toff += K
    return np.concatenate(Hs), np.array(h_off), np.array(t_off), toff


@pytest.mark.parametrize("graphs", [False, True])
def test_uneven_batch_matches_uniform_and_oracle(orc, graphs):
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan, inst_table
    B, T = 600, 10
    shapes = ch.uneven_shapes(B, seed=3)
    Hflat, h_off, t_off, nt = pack(shapes, seed=3)
    tflat = np.ones(nt, np.float32)
    mu = ch.uniform_steps(T, 0.01, 0.1, seed=2)
    plan = Plan(capi.LAYER_PROJ, T, [tuple(s) for s in ch.UNEVEN_SHAPES], B, graphs=graphs)
    tbl = inst_table(h_off, h_off, t_off, shapes[:, 0], shapes[:, 1]).cuda()
    Hd = torch.from_numpy(Hflat).cuda()
    td = torch.from_numpy(tflat).cuda()
    md = torch.from_numpy(mu).cuda()
    for rep in range(2):  # second call re-arms the graph
        W, obj, res, fl = plan.solve_varlen(tbl, Hd, td, md)
        torch.cuda.synchronize()
    W, obj, res, fl = W.cpu().numpy(), obj.cpu().numpy(), res.cpu().numpy(), fl.cpu().numpy()
    assert np.all(fl[fl != 0] == capi.F_FP64_CHOL)
    for (M, K) in ch.UNEVEN_SHAPES:
        idx = np.where((shapes[:, 0] == M) & (shapes[:, 1] == K))[0]
        assert len(idx) > 50
        Hb = np.stack([Hflat[h_off[b]:h_off[b] + K * M].reshape(K, M) for b in idx])
        Wu, ou, _, fu = plan.solve(torch.from_numpy(Hb).cuda(), torch.ones(K, device="cuda"), md)
        Wv = np.stack([W[h_off[b]:h_off[b] + K * M].reshape(K, M) for b in idx])
        assert np.array_equal(Wv, Wu.cpu().numpy()), (M, K)
        assert np.array_equal(obj[idx], ou.cpu().numpy())
        sel = idx[:24]
        Hs = np.stack([Hflat[h_off[b]:h_off[b] + K * M].reshape(K, M) for b in sel])
        Wo, oo, ro, so = orc.batch_forward(1, Hs.astype(np.complex128), np.ones((len(sel), K)),
                                           mu.astype(np.float64), nthreads=8)
        Wg = np.stack([W[h_off[b]:h_off[b] + K * M].reshape(K, M) for b in sel])
        err = np.linalg.norm((Wg - Wo).reshape(len(sel), -1), axis=1) / np.linalg.norm(
            Wo.reshape(len(sel), -1), axis=1)
        assert err.max() <= 1e-4, (M, K, err.max())
        assert np.max(np.abs(obj[sel] - oo) / oo) <= 1e-5
    plan.close()


def test_uneven_tensor_core_buckets_with_padded_users(orc):
    """Serving-like shapes on a tensor-core plan: M in {64, 128, 256} with any K
    (user-padded tensor-core buckets) plus shapes only the FP32 generic buckets
    hold (M = 100).  Every instance equals the uniform solve of its shape and
    matches the FP64 oracle."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan, inst_table
    rs = np.random.default_rng(4)
    B, T = 400, 10
    M = rs.choice([64, 128, 256], B)
    K = rs.integers(4, 33, B)
    M[:12] = 100
    shapes = np.stack([M, K], 1).astype(np.int32)
    Hflat, h_off, t_off, nt = pack(shapes, seed=4)
    tflat = np.ones(nt, np.float32)
    mu = ch.uniform_steps(T, 0.01, 0.1, seed=2)
    bucket_shapes = [(m, k) for m in (64, 128, 256) for k in (8, 16, 24, 32)]
    plan = Plan(capi.LAYER_PROJ, T, bucket_shapes, B, graphs=True, tensor_cores=True)
    tbl = inst_table(h_off, h_off, t_off, shapes[:, 0], shapes[:, 1]).cuda()
    Hd = torch.from_numpy(Hflat).cuda()
    td = torch.from_numpy(tflat).cuda()
    md = torch.from_numpy(mu).cuda()
    W, obj, res, fl = plan.solve_varlen(tbl, Hd, td, md)
    torch.cuda.synchronize()
    W, obj, fl = W.cpu().numpy(), obj.cpu().numpy(), fl.cpu().numpy()
    assert np.all(fl[fl != 0] == capi.F_FP64_CHOL)
    for (m, k) in {(int(a), int(b)) for a, b in shapes}:
        idx = np.where((shapes[:, 0] == m) & (shapes[:, 1] == k))[0]
        Hb = np.stack([Hflat[h_off[b]:h_off[b] + k * m].reshape(k, m) for b in idx])
        Wo, oo, ro, so = orc.batch_forward(1, Hb.astype(np.complex128), np.ones((len(idx), k)),
                                           mu.astype(np.float64), nthreads=8)
        Wg = np.stack([W[h_off[b]:h_off[b] + k * m].reshape(k, m) for b in idx])
        err = np.linalg.norm((Wg - Wo).reshape(len(idx), -1), axis=1) / np.linalg.norm(
            Wo.reshape(len(idx), -1), axis=1)
        # every instance, FP64-path ones included (they run in an orthonormal basis
        # of the channel's row space), at the same bar
        assert err.max() <= 1e-4, (m, k, err.max(), fl[idx][err.argmax()])
        assert np.max(np.abs(obj[idx] - oo) / oo) <= 1e-5, (m, k)
        if m != 100:
            pu = Plan(capi.LAYER_PROJ, T, [(m, k)], len(idx), tensor_cores=True)
            Wu, ou, _, _ = pu.solve(torch.from_numpy(Hb).cuda(), torch.ones(k, device="cuda"), md)
            assert np.array_equal(Wg, Wu.cpu().numpy()), (m, k)
            assert capi.precode_plan_describe(pu.handle, m, k).startswith(("solve_tc", "solve_tg")), (m, k)
            pu.close()
    plan.close()


def test_uneven_batch_rejects_bad_descriptors(orc):
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan, inst_table
    shapes = np.array([[64, 8], [63, 8], [64, 8], [16, 20], [64, 8], [300, 8]], np.int32)
    Hflat, h_off, t_off, nt = pack([(64, 8)] * len(shapes), seed=9)
    h_off = h_off.copy()
    h_off[2] += 1  # odd offset: misaligned instance
    plan = Plan(capi.LAYER_PROJ, 4, [(64, 8)], 8, graphs=True)
    tbl = inst_table(h_off, h_off, t_off, shapes[:, 0], shapes[:, 1]).cuda()
    W, obj, res, fl = plan.solve_varlen(tbl, torch.from_numpy(Hflat).cuda(),
                                        torch.ones(nt, device="cuda"),
                                        torch.full((4,), 0.05, device="cuda"))
    fl = fl.cpu().numpy()
    assert list(fl == capi.F_INVALID) == [False, True, True, True, False, True]
    good = [0, 4]
    Hs = np.stack([Hflat[h_off[b]:h_off[b] + 512].reshape(8, 64) for b in good])
    Wo, oo, _, _ = orc.batch_forward(1, Hs.astype(np.complex128), np.ones((2, 8)), [0.05] * 4)
    Wg = W.cpu().numpy()
    for i, b in enumerate(good):
        Wb = Wg[h_off[b]:h_off[b] + 512].reshape(8, 64)
        assert np.linalg.norm(Wb - Wo[i]) / np.linalg.norm(Wo[i]) <= 1e-4
    plan.close()
