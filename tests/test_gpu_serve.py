"""Continuous-batching server: correctness, alone-vs-mix equality, resident channels."""
import threading

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_12745_gb300 import channels as ch

pytestmark = pytest.mark.gpu

SHAPES = [(32, 4), (64, 8), (128, 16), (256, 32)]
# the benchmark's serving configuration: every job shape (M in {64, 128, 256}, any
# K <= 32) fits a user-padded tensor-core bucket of 8, 16, 24 or 32 users
BENCH_SHAPES = [(m, k) for m in (64, 128, 256) for k in (8, 16, 24, 32)]


@pytest.fixture(scope="module", params=["fp32_buckets", "tensor_core_buckets"])
def server(request):
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.serving import Server
    mu = ch.uniform_steps(10, 0.01, 0.1, seed=2)
    if request.param == "fp32_buckets":
        s = Server(capi.LAYER_PROJ, mu, shapes=SHAPES, n_slots=4, max_batch_instances=8192,
                   device_mem_budget=1 << 30)
    else:  # as bench.py's serving workload builds it
        s = Server(capi.LAYER_PROJ, mu, shapes=BENCH_SHAPES, n_slots=6, max_batch_instances=65536,
                   device_mem_budget=4 << 30, flags=capi.PLAN_TENSOR_CORES)
    s.kind = request.param
    yield s, mu
    s.close()


def test_jobs_match_oracle(orc, server):
    """Jobs of the serving workload's shapes (M in {64, 128, 256}, K in 4..32,
    Rician), every subcarrier of every job against the FP64 oracle."""
    s, mu = server
    rng = np.random.default_rng(0)
    jobs = []
    for i in range(12):
        M = int(rng.choice([64, 128, 256]))
        K = int(rng.integers(4, 33))
        H = ch.rician_ula(int(rng.choice([16, 64])), K, M, seed=100 + i)
        jobs.append((H, s.submit(H, np.ones(K, np.float32))))
    for H, h in jobs:
        r = h.wait()
        assert r.status == 0 and r.latency_us > 0
        n, K, M = H.shape
        Wo, oo, _, so = orc.batch_forward(1, H.astype(np.complex128), np.ones((n, K)),
                                          mu.astype(np.float64), nthreads=8)
        assert np.all(so == 0) and np.all(h.flags == 0)
        err = np.linalg.norm((h.W - Wo).reshape(n, -1), axis=1) / np.linalg.norm(Wo.reshape(n, -1), axis=1)
        assert err.max() <= 1e-4, (M, K, err.max())
        assert np.max(np.abs(h.obj - oo) / oo) <= 1e-5, (M, K)


def test_result_same_alone_and_in_the_mix(server):
    s, mu = server
    H = ch.rician_ula(256, 12, 128, seed=7)
    t = np.ones(12, np.float32)
    alone = s.submit(H, t)
    alone.wait()
    W_alone, obj_alone = alone.W.copy(), alone.obj.copy()
    # now the same job among many others submitted concurrently from 4 threads
    rng = np.random.default_rng(1)
    others = [ch.rician_ula(int(rng.choice([64, 256, 512])), int(rng.integers(4, 33)),
                            int(rng.choice([64, 128, 256])), seed=200 + i) for i in range(24)]
    handles, lock = [], threading.Lock()

    def worker(chunk):
        for H2 in chunk:
            h = s.submit(H2, np.ones(H2.shape[1], np.float32))
            with lock:
                handles.append(h)

    threads = [threading.Thread(target=worker, args=(others[i::4],)) for i in range(4)]
    for th in threads:
        th.start()
    mixed = s.submit(H, t)
    for th in threads:
        th.join()
    mixed.wait()
    for h in handles:
        assert h.wait().status == 0
    st = s.stats()
    assert st["launches"] >= 2
    assert np.array_equal(mixed.W, W_alone) and np.array_equal(mixed.obj, obj_alone)


def test_resident_channel_matches_copied_channel(server):
    s, mu = server
    H = ch.rician_ula(128, 8, 64, seed=9)
    t = np.ones(8, np.float32)
    cid = s.channel(H)
    a = s.submit(H, t)
    b = s.submit(None, t, channel=cid, M=64, K=8, n_sc=128)
    a.wait()
    b.wait()
    assert np.array_equal(a.W, b.W)
    s.release_channel(cid)


@pytest.mark.parametrize("M,K", [(64, 8), (128, 16), (256, 32), (256, 20)])
def test_resident_factors_bitwise_and_parity(orc, server, M, K):
    """A resident channel on the tensor-core buckets keeps each subcarrier's Gram
    inverse (split-FP16 K = 8, multi-warp split-FP16 and tcgen05 kernels): jobs on it
    give bitwise the copied channel's results, match the oracle, and are counted as
    launched with factors.  Every fourth subcarrier has a near-collinear user pair
    (FP64 path: no factor, set up in full by every job)."""
    from paper_2304_12745_gb300 import capi
    s, mu = server
    if s.kind != "tensor_core_buckets":  # the FFMA buckets keep no factors
        pytest.skip("the tensor-core bucket server only")
    n = 96
    H = ch.rician_ula(n, K, M, seed=300 + K)
    rs = np.random.default_rng(301)
    for b in range(0, n, 4):
        H[b, 1] = H[b, 0] + (1e-4 * (rs.standard_normal(M) + 1j * rs.standard_normal(M))).astype(np.complex64)
    t = np.ones(K, np.float32)
    cid = s.channel(H)
    f0 = s.stats()["factor_instances"]
    a = s.submit(H, t)
    b = s.submit(None, t, channel=cid, M=M, K=K, n_sc=n)
    a.wait()
    b.wait()
    assert s.stats()["factor_instances"] - f0 == n
    assert np.array_equal(a.W, b.W) and np.array_equal(a.obj, b.obj) and np.array_equal(a.flags, b.flags)
    assert np.all(b.flags[0::4] == capi.F_FP64_CHOL) and np.all((b.flags == 0) | (b.flags == capi.F_FP64_CHOL))
    Wo, oo, _, so = orc.batch_forward(1, H.astype(np.complex128), np.ones((n, K)),
                                      mu.astype(np.float64), nthreads=8)
    err = np.linalg.norm((b.W - Wo).reshape(n, -1), axis=1) / np.linalg.norm(Wo.reshape(n, -1), axis=1)
    assert err.max() <= 1e-4, err.max()
    assert np.max(np.abs(b.obj - oo) / oo) <= 1e-5
    s.release_channel(cid)


def test_poisson_load_reports_latency():
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.serving import Server, poisson_load
    mu = ch.uniform_steps(10, 0.01, 0.1, seed=2)
    s = Server(capi.LAYER_PROJ, mu, shapes=SHAPES, n_slots=4, max_batch_instances=16384,
               device_mem_budget=4 << 30)
    st = poisson_load(s, rate_per_s=500.0, duration_s=0.5, seed=3, nsc_choices=(64, 128, 256))
    s.close()
    assert st["completed"] == st["jobs"] > 100
    assert 0 < st["p50_us"] <= st["p99_us"] <= st["max_us"]
    assert st["precoders_per_s"] > 0
