"""Failure detection without a GPU fault.

* Device-side waits: the kernels' bounded wait for an instance's channel copy is
  shortened through the plan and made to run out by issuing no copy at all
  (``precode_plan_set_debug``: nothing is in flight, so nothing faults or
  hangs); the instance reaches the caller as ``PRECODE_F_TIMEOUT`` and the plan's
  error counter, and the context stays usable: the same plan solves correctly
  afterwards.
* Allocation failure: ``PRECODE_INJECT_ENOMEM=N`` makes the library's N-th
  device or page-locked allocation fail; plans and servers return
  ``PRECODE_ENOMEM`` from whichever allocation that is, and free what they held.
* Host waits: ``precode_serve_wait`` with a limit shorter than the job returns
  ``PRECODE_ETIMEDOUT`` and the job still completes.
"""
import os
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_12745_gb300 import channels as ch

pytestmark = pytest.mark.gpu

SENTINEL = -12345


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12745_gb300 import capi, precoder
    return capi, precoder


# (label, M, K, plan options): the FFMA kernel, the one-warp split-FP16 kernel, the
# multi-warp split-FP16 kernel and the two tcgen05 builds (named by their key)
STALL_CASES = [("ffma", 32, 4, {}), ("tch", 64, 8, dict(tensor_cores=True)),
               ("tcwh", 256, 32, dict(tensor_cores=True)), ("tg", 256, 32, "tg"),
               ("tgt", 256, 32, "tgt")]


def tg_build(tmp_path, capi, M, K, suffix):
    """Plan options that pin (M, K) to a tcgen05 build (the row build, key suffix
    "tg", or the transposed one, "tg/tgt")."""
    path = tmp_path / "tune_tg.txt"
    path.write_text(f"{torch.cuda.get_device_name(0)}|{capi.LAYER_PROJ}|{K}|{M}\t"
                    f"32x256/4x8/jc8/w8/b1/split/tc/f16/{suffix}/generic\n")
    return dict(tensor_cores=True, autotune=True, tune_cache=str(path))


@pytest.mark.parametrize("label,M,K,kw", STALL_CASES)
def test_copy_wait_runs_out_and_is_reported(pc, orc, tmp_path, label, M, K, kw):
    capi, precoder = pc
    if isinstance(kw, str):
        kw = tg_build(tmp_path, capi, M, K, "tg" if kw == "tg" else "tg/tgt")
    B, T = 96, 4
    H = ch.rayleigh(B, K, M, seed=80 + K)
    t = ch.targets(B, K)
    mu = np.full(T, 0.05, np.float32)
    plan = precoder.Plan(capi.LAYER_PROJ, T, [(M, K)], B, **kw)
    Hd, td, md = torch.from_numpy(H).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(mu).cuda()
    out = (torch.zeros_like(Hd), torch.zeros(B, device="cuda"), torch.zeros(B, device="cuda"),
           torch.full((B,), SENTINEL, dtype=torch.int32, device="cuda"))
    capi.precode_plan_set_debug(plan.handle, 200_000, True)  # 0.2 ms limit, no copies issued
    t0 = time.perf_counter()
    plan.solve(Hd, td, md, out=out)
    torch.cuda.synchronize()
    elapsed = time.perf_counter() - t0
    fl = out[3].cpu().numpy()
    n_err = plan.errors()
    # every group / block reports the instance it was waiting for, then gives up
    assert np.any(fl == capi.F_TIMEOUT)
    assert np.all((fl == capi.F_TIMEOUT) | (fl == SENTINEL))
    assert n_err == int((fl == capi.F_TIMEOUT).sum())
    assert not torch.any(out[0]).item()  # no W written
    assert elapsed < 5.0
    # normal operation again on the same plan and context
    capi.precode_plan_set_debug(plan.handle, 0, False)
    W, obj, res, fl2 = plan.solve(Hd, td, md)
    torch.cuda.synchronize()
    assert plan.errors() == n_err
    assert np.all(fl2.cpu().numpy() == 0)
    Wo, oo, _, _ = orc.batch_forward(1, H.astype(np.complex128), t.astype(np.float64),
                                     mu.astype(np.float64), nthreads=8)
    Wg = W.cpu().numpy()
    err = np.linalg.norm((Wg - Wo).reshape(B, -1), axis=1) / np.linalg.norm(Wo.reshape(B, -1), axis=1)
    assert err.max() <= 1e-4
    plan.close()


def test_copy_wait_runs_out_in_uneven_batch_and_train_step(pc):
    capi, precoder = pc
    from paper_2304_12745_gb300.precoder import inst_table
    shapes = [(64, 8)] * 20 + [(32, 4)] * 12
    sizes = [m * k for m, k in shapes]
    h_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    t_off = np.concatenate([[0], np.cumsum([k for _, k in shapes])[:-1]]).astype(np.int64)
    Hflat = np.concatenate([ch.rayleigh(1, k, m, seed=90 + i).reshape(-1)
                            for i, (m, k) in enumerate(shapes)]).astype(np.complex64)
    plan = precoder.Plan(capi.LAYER_PROJ, 4, [(64, 8), (32, 4)], len(shapes), graphs=True,
                         tensor_cores=True)
    tbl = inst_table(h_off, h_off, t_off, [m for m, _ in shapes], [k for _, k in shapes]).cuda()
    Hd = torch.from_numpy(Hflat).cuda()
    td = torch.ones(int(sum(k for _, k in shapes)), device="cuda")
    md = torch.full((4,), 0.05, device="cuda")
    W, obj, res, fl = plan.solve_varlen(tbl, Hd, td, md)  # builds the graph
    torch.cuda.synchronize()
    assert np.all(fl.cpu().numpy() == 0)
    capi.precode_plan_set_debug(plan.handle, 200_000, True)
    fl = plan.solve_varlen(tbl, Hd, td, md)[3]  # the graph re-armed with the stall
    torch.cuda.synchronize()
    f = fl.cpu().numpy()  # flags start at 0; unreached instances keep it
    assert np.any(f == capi.F_TIMEOUT) and np.all((f == capi.F_TIMEOUT) | (f == 0))
    assert plan.errors() == int((f == capi.F_TIMEOUT).sum())
    capi.precode_plan_set_debug(plan.handle, 0, False)
    fl = plan.solve_varlen(tbl, Hd, td, md)[3]
    torch.cuda.synchronize()
    assert np.all(fl.cpu().numpy() == 0)
    plan.close()

    # train step: the forward's copy wait
    B, K, M, T = 64, 8, 64, 4
    tp = precoder.Plan(capi.LAYER_PROJ, T, [(M, K)], B, tensor_cores=True)
    Ht = torch.from_numpy(ch.rayleigh(B, K, M, seed=95)).cuda()
    tt = torch.ones(K, device="cuda")
    mu = torch.full((T,), 0.05, device="cuda")
    loss, dmu = torch.empty(1, device="cuda"), torch.empty(T, device="cuda")
    flt = torch.full((B,), SENTINEL, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    capi.precode_train_step(tp.handle, M, K, B, Ht, tt, 0, mu, None, 1.0, loss, dmu, None, None, stream)
    torch.cuda.synchronize()
    capi.precode_plan_set_debug(tp.handle, 200_000, True)
    capi.precode_train_step(tp.handle, M, K, B, Ht, tt, 0, mu, None, 1.0, loss, dmu, None, flt, stream)
    torch.cuda.synchronize()
    f = flt.cpu().numpy()
    assert np.any(f == capi.F_TIMEOUT) and tp.errors() >= 1
    capi.precode_plan_set_debug(tp.handle, 0, False)
    flt.fill_(SENTINEL)
    capi.precode_train_step(tp.handle, M, K, B, Ht, tt, 0, mu, None, 1.0, loss, dmu, None, flt, stream)
    torch.cuda.synchronize()
    assert np.all(flt.cpu().numpy() == 0) and np.isfinite(float(loss))
    tp.close()


def _with_enomem(n, fn):
    os.environ["PRECODE_INJECT_ENOMEM"] = str(n)
    try:
        return fn()
    finally:
        del os.environ["PRECODE_INJECT_ENOMEM"]


def test_injected_allocation_failure_plan_and_server(pc):
    capi, precoder = pc
    shapes = [(64, 8), (256, 32)]

    def make_plan():
        return precoder.Plan(capi.LAYER_PROJ, 4, shapes, 1024, tensor_cores=True)

    def make_server():
        from paper_2304_12745_gb300.serving import Server
        return Server(capi.LAYER_PROJ, np.full(4, 0.05, np.float32), shapes=shapes, n_slots=2,
                      max_batch_instances=1024, device_mem_budget=64 << 20,
                      flags=capi.PLAN_TENSOR_CORES)

    for make in (make_plan, make_server):
        failed = 0
        for n in range(1, 40):
            try:
                obj = _with_enomem(n, make)
            except capi.PrecodeError as e:
                assert e.status == capi.ENOMEM, (make.__name__, n, e)
                failed += 1
                continue
            obj.close()  # fewer than n allocations: it succeeded
            break
        else:
            pytest.fail(f"{make.__name__} still failing after 39 injected failures")
        assert failed >= 1, make.__name__
    # nothing left behind: a plan works normally
    p = make_plan()
    H = torch.from_numpy(ch.rayleigh(8, 8, 64, seed=3)).cuda()
    W, obj, res, fl = p.solve(H, torch.ones(8, device="cuda"), torch.full((4,), 0.05, device="cuda"))
    torch.cuda.synchronize()
    assert np.all(fl.cpu().numpy() == 0) and torch.isfinite(obj).all()
    p.close()


def test_serve_wait_times_out_then_completes(pc):
    """A long job (1,024 subcarriers of 32 x 256, 2,000 layers, one slot) is still
    running when a 1 ms wait on it ends: ETIMEDOUT; the job then completes."""
    capi, _ = pc
    from paper_2304_12745_gb300 import serving
    K, M, T, n_sc = 32, 256, 2000, 1024
    s = serving.Server(capi.LAYER_PROJ, np.full(T, 0.02, np.float32), shapes=[(M, K)], n_slots=1,
                       max_batch_instances=n_sc, device_mem_budget=1 << 30,
                       flags=capi.PLAN_TENSOR_CORES)
    H = ch.rician_ula(n_sc, K, M, seed=7)
    job = s.submit(H, np.ones(K, np.float32))
    with pytest.raises(capi.PrecodeError) as ei:
        job.wait(timeout_us=1000)
    assert ei.value.status == capi.ETIMEDOUT
    r = job.wait()
    assert r.status == capi.OK and r.latency_us > 1000
    assert np.isfinite(job.W).all() and np.all(job.flags == 0)
    s.close()
