"""Host buffers on the paper layer at K = 8, M = 64 (split-FP16 build).

The zero-copy host-buffer kernels are projected-layer builds, so a paper-layer
plan takes the staged copy pipeline whether the buffers are page-locked or not;
both must give bitwise the device solve's outputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_12745_gb300 import channels as ch

pytestmark = pytest.mark.gpu


def test_paper_layer_host_buffers_match_device_solve():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12745_gb300 import capi, precoder
    B, K, M, T = 5003, 8, 64, 10
    H = ch.rayleigh(B, K, M, seed=43)
    t = ch.targets(B, K, gamma_db=10.0)
    eta = np.full(T, ch.paper_eta(K, M), np.float32)
    lam = np.full(T, 1 / 15, np.float32)
    plan = precoder.Plan(capi.LAYER_PGD, T, [(M, K)], B, tensor_cores=True)
    assert capi.precode_plan_describe(plan.handle, M, K).startswith("solve_tch_kernel")
    a = plan.solve(torch.from_numpy(H).cuda(), torch.from_numpy(t).cuda(),
                   torch.from_numpy(eta).cuda(), torch.from_numpy(lam).cuda())
    a = [x.cpu() for x in a]
    for pinned in (True, False):
        def buf(x):
            return x.pin_memory() if pinned else x
        Hh, th = buf(torch.from_numpy(H)), buf(torch.from_numpy(t))
        Wh = buf(torch.empty(B, K, M, dtype=torch.complex64))
        oh, rh = buf(torch.empty(B)), buf(torch.empty(B))
        fh = buf(torch.empty(B, dtype=torch.int32))
        plan.solve_host(Hh, th, torch.from_numpy(eta), torch.from_numpy(lam), W=Wh, obj=oh,
                        resid=rh, flags=fh)
        assert torch.equal(Wh, a[0]) and torch.equal(oh, a[1]), pinned
        assert torch.equal(rh, a[2]) and torch.equal(fh, a[3]), pinned
    assert plan.errors() == 0
    plan.close()
