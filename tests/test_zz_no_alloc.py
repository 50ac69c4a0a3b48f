"""The allocation-free uneven-batch entry point, against the plan-based one.

precode_solve_varlen_static exists for callers that may not allocate device
memory while they run (for example a real-time baseband loop that reserves
everything at start-up): it keeps its scratch in a fixed array inside the
library instead of plan workspace.  This test calls it through the C ABI
twice in a row on different uneven batches, and checks each result against
precode_solve_varlen with a plan of the same shapes: both run the same kernel
variants, so W, the objective, the residual and the flags agree bit for bit
(which implies the parity tolerances used elsewhere).  The second call checks
that the shared scratch is cleared between calls.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_12745_gb300 import channels as ch

pytestmark = pytest.mark.gpu

def _uneven_batch(B, seed):
    shapes = ch.uneven_shapes(B, seed=seed)
    Hs, h_off, t_off, off, toff = [], [], [], 0, 0
    for b, (M, K) in enumerate(shapes):
        H = ch.rician_ula(1, int(K), int(M), seed=seed * 7919 + b)[0]
        Hs.append(H.reshape(-1))
        h_off.append(off)
        t_off.append(toff)
        off += H.size
        toff += int(K)
    h_off = np.array(h_off)
    h_off_bad = h_off.copy()
    h_off_bad[5] += 1  # one misaligned descriptor: both paths must reject it
    return shapes, np.concatenate(Hs), h_off, h_off_bad, np.array(t_off), toff


def test_static_scratch_entry_point_matches_plan_path():
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan, inst_table
    assert torch.cuda.is_available()
    T = 10
    mu = torch.from_numpy(ch.uniform_steps(T, 0.01, 0.1, seed=2)).cuda()
    plan_shapes = [tuple(s) for s in ch.UNEVEN_SHAPES]
    stream = torch.cuda.current_stream().cuda_stream
    for call, (B, seed) in enumerate([(400, 21), (250, 22)]):
        shapes, Hflat, h_off, h_bad, t_off, nt = _uneven_batch(B, seed)
        tbl = inst_table(h_bad, h_off, t_off, shapes[:, 0], shapes[:, 1]).cuda()
        Hd = torch.from_numpy(Hflat).cuda()
        td = torch.ones(nt, device="cuda")
        plan = Plan(capi.LAYER_PROJ, T, plan_shapes, B)
        Wp, op, rp, fp = plan.solve_varlen(tbl, Hd, td, mu)
        Ws = torch.zeros_like(Hd)
        od = torch.empty(B, device="cuda")
        rs = torch.empty(B, device="cuda")
        fs = torch.zeros(B, device="cuda", dtype=torch.int32)
        capi.precode_solve_varlen_static(capi.LAYER_PROJ, T, plan_shapes, B, tbl, Hd, td, mu, None,
                                         Ws, od, rs, fs, stream)
        torch.cuda.synchronize()
        plan.close()
        fp, fsn = fp.cpu().numpy(), fs.cpu().numpy()
        assert np.array_equal(fp, fsn), f"call {call}: flags differ"
        assert fsn[5] == capi.F_INVALID and (fsn != capi.F_INVALID).sum() == B - 1
        Wp, Wn = Wp.cpu().numpy(), Ws.cpu().numpy()
        op, os_ = op.cpu().numpy(), od.cpu().numpy()
        rp, rs_ = rp.cpu().numpy(), rs.cpu().numpy()
        ok = np.arange(B) != 5
        assert np.array_equal(os_[ok], op[ok]) and np.array_equal(rs_[ok], rp[ok]), call
        for b in range(B):
            if b == 5:
                continue
            K, M = int(shapes[b, 1]), int(shapes[b, 0])
            a = Wn[h_off[b]:h_off[b] + K * M]
            r = Wp[h_off[b]:h_off[b] + K * M]
            assert np.array_equal(a, r), (call, b)
    # sizes beyond the fixed scratch are refused before anything runs
    with pytest.raises(capi.PrecodeError) as ex:
        capi.precode_solve_varlen_static(capi.LAYER_PROJ, T, plan_shapes, 65537, tbl, Hd, td, mu,
                                         None, Ws, od, rs, fs, stream)
    assert ex.value.status == capi.EINVAL
    # tensor-core buckets need a plan: refused, not silently run on the FP32 variants
    with pytest.raises(capi.PrecodeError) as ex:
        capi.precode_solve_varlen_static(capi.LAYER_PROJ, T, plan_shapes, 10, tbl, Hd, td, mu,
                                         None, Ws, od, rs, fs, stream,
                                         flags_desc=capi.PLAN_TENSOR_CORES)
    assert ex.value.status == capi.EINVAL
