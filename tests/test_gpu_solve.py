"""GPU parity of the batched solve (both layer maps) against the FP64 oracle.

Bar (per instance): relative Frobenius error of W <= 1e-4 and relative error
of the objective ||W||_{2,1} <= 1e-5, on the same seeded inputs; integer
outputs (flags) exact.  Inputs follow the benchmark workloads: i.i.d. CN(0,1)
and log-normal-scaled Rayleigh channels, Rician ULA channels for the larger
buckets, unit targets or the paper's 10 dB targets.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_12745_gb300 import channels as ch

pytestmark = pytest.mark.gpu

W_TOL = 1e-4
OBJ_TOL = 1e-5


@pytest.fixture(scope="module")
def pc():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2304_12745_gb300 import capi, precoder
    return capi, precoder


def run_gpu(precoder, mode, H, t, step, lam=None, **plan_kw):
    B, K, M = H.shape
    plan = precoder.Plan(mode, len(step), [(M, K)], max(B, 1), **plan_kw)
    Hd = torch.from_numpy(H).cuda()
    td = torch.from_numpy(np.ascontiguousarray(t, dtype=np.float32)).cuda()
    sd = torch.tensor(step, dtype=torch.float32, device="cuda")
    ld = torch.tensor(lam, dtype=torch.float32, device="cuda") if lam is not None else None
    W, obj, res, fl = plan.solve(Hd, td, sd, ld)
    torch.cuda.synchronize()
    assert plan.errors() == 0
    out = W.cpu().numpy(), obj.cpu().numpy(), res.cpu().numpy(), fl.cpu().numpy()
    plan.close()
    return out


def oracle_ref(orc, mode, H, t, step, lam=None):
    B, K, M = H.shape
    tt = np.broadcast_to(np.asarray(t, np.float64), (B, K))
    return orc.batch_forward(mode, H.astype(np.complex128), tt, np.asarray(step, np.float64),
                             None if lam is None else np.asarray(lam, np.float64), nthreads=8)


def rel_fro(A, B):
    num = np.linalg.norm((A - B).reshape(len(A), -1), axis=1)
    den = np.maximum(np.linalg.norm(B.reshape(len(B), -1), axis=1), 1e-30)
    return num / den


def assert_parity(gpu, ref, w_tol=W_TOL, obj_tol=OBJ_TOL, resid_abs=None):
    Wg, og, rg, fg = gpu
    Wo, oo, ro, so = ref
    e = rel_fro(Wg, Wo)
    assert e.max() <= w_tol, f"max rel-Fro error {e.max():.3e} at instance {e.argmax()}"
    eo = np.abs(og - oo) / np.maximum(oo, 1e-30)
    assert eo.max() <= obj_tol, f"max objective error {eo.max():.3e} at {eo.argmax()}"
    if resid_abs is not None:
        assert np.all(rg <= resid_abs)
    return e, eo


# ---------------------------------------------------------------- projected layer

def test_proj_tiny_workload(pc, orc):
    """128 x C^{4x32} CN(0,1), unit targets, T = 20, mu_t = 0.05."""
    capi, precoder = pc
    H = ch.rayleigh(128, 4, 32, seed=1)
    t = ch.targets(128, 4)
    mu = np.full(20, 0.05, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu)
    ref = oracle_ref(orc, 1, H, t, mu)
    assert_parity(gpu, ref, resid_abs=1e-4)
    assert np.all(gpu[3] == 0)


def test_proj_fixed_workload_sample(pc, orc):
    """C^{8x64}, 8 dB log-normal user gains, T = 10, mu_t ~ U[0.01, 0.1] (seed 2);
    a ragged batch of 1000 instances."""
    capi, precoder = pc
    H = ch.lognormal(1000, 8, 64, seed=2)
    t = ch.targets(1000, 8)
    mu = ch.fixed_workload_steps(10)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu)
    ref = oracle_ref(orc, 1, H, t, mu)
    assert_parity(gpu, ref)
    # residual of a feasible output is rounding-level relative to ||S||_F
    assert np.all(gpu[2] <= 1e-4 * math.sqrt(8))


def test_proj_paper_targets_and_sum_rate(pc, orc):
    """10 dB targets (t = sqrt(10)), K=8, M=64: every output is feasible, so the
    sum rate equals the paper's 27.68 bits/symbol."""
    capi, precoder = pc
    H = ch.rayleigh(64, 8, 64, seed=3)
    t = ch.targets(64, 8, gamma_db=10.0)
    mu = np.full(10, 0.3, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu)
    ref = oracle_ref(orc, 1, H, t, mu)
    assert_parity(gpu, ref)
    for b in range(0, 64, 9):
        r = orc.sum_rate(H[b].astype(np.complex128), gpu[0][b].astype(np.complex128), 1.0)
        assert abs(r - 8 * math.log2(1 + float(t[b, 0]) ** 2)) < 1e-3


@pytest.mark.parametrize("K,M", [(16, 128), (32, 256)])
def test_proj_large_buckets(pc, orc, K, M):
    capi, precoder = pc
    B = 96
    H = ch.rician_ula(B, K, M, seed=5)
    t = ch.targets(B, K)
    mu = ch.uniform_steps(10, 0.01, 0.1, seed=7)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu)
    ref = oracle_ref(orc, 1, H, t, mu)
    assert_parity(gpu, ref)


@pytest.mark.parametrize("K,M", [(3, 20), (4, 4), (5, 40), (8, 10), (11, 100), (32, 200)])
def test_proj_generic_buckets(pc, orc, K, M):
    """Shapes that only fit a larger bucket (runtime K, M); M = K leaves no freedom."""
    capi, precoder = pc
    B = 37
    H = ch.rayleigh(B, K, M, seed=11 + K)
    t = ch.targets(B, K)
    mu = np.full(6, 0.05, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu)
    ref = oracle_ref(orc, 1, H, t, mu)
    assert_parity(gpu, ref)
    if M == K:
        for b in range(B):
            Wstar = np.linalg.solve(H[b].astype(np.complex128), np.diag(t[b]).astype(np.complex128)).T
            assert np.linalg.norm(gpu[0][b] - Wstar) / np.linalg.norm(Wstar) < W_TOL


def test_proj_singular_and_nonfinite_flags(pc, orc):
    capi, precoder = pc
    H = ch.rayleigh(8, 4, 32, seed=21)
    H[2, 3] = H[2, 1]          # rank 3: singular Gram
    H[5, 0, 7] = np.nan        # non-finite input
    t = ch.targets(8, 4)
    mu = np.full(5, 0.05, np.float32)
    W, obj, res, fl = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu)
    assert fl[2] & capi.F_SINGULAR and fl[2] & capi.F_FP64_CHOL
    assert not np.any(W[2]) and obj[2] == 0
    assert res[2] == pytest.approx(2.0, rel=1e-6)  # ||S||_F with W = 0
    assert fl[5] & capi.F_NONFINITE
    ok = [0, 1, 3, 4, 6, 7]
    assert np.all(fl[ok] == 0)
    ref = oracle_ref(orc, 1, H[ok], t[ok], mu)
    assert_parity((W[ok], obj[ok], res[ok], fl[ok]), ref)


def test_proj_ill_conditioned_uses_fp64(pc, orc):
    """Two almost collinear users push the equilibrated pivot ratio over the
    threshold: the FP64 path runs (Gram factorised in FP64, the layers in an
    orthonormal basis of the channel's row space) and the FP32 bar still holds."""
    capi, precoder = pc
    rs = np.random.default_rng(5)
    H = ch.rayleigh(16, 4, 32, seed=22)
    for b in range(0, 16, 2):
        H[b, 1] = H[b, 0] + (1e-3 * (rs.standard_normal(32) + 1j * rs.standard_normal(32))).astype(np.complex64)
    t = ch.targets(16, 4)
    mu = np.full(4, 0.02, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, cond_threshold=1e3)
    assert np.all(gpu[3][0::2] == capi.F_FP64_CHOL)
    assert np.all(gpu[3][1::2] == 0)
    ref = oracle_ref(orc, 1, H, t, mu)
    assert_parity(gpu, ref)


# ---------------------------------------------------------------- paper layer

def test_pgd_tiny_workload_paper_parameters(pc, orc):
    """Paper layer on 128 x C^{4x32}: eta = 1/L~ (Marchenko-Pastur edge), lambda = 1/15, T = 20."""
    capi, precoder = pc
    H = ch.rayleigh(128, 4, 32, seed=1)
    t = ch.targets(128, 4)
    eta = np.full(20, ch.paper_eta(4, 32), np.float32)
    lam = np.full(20, 1 / 15, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PGD, H, t, eta, lam)
    ref = oracle_ref(orc, 0, H, t, eta, lam)
    assert_parity(gpu, ref)
    eo = np.abs(gpu[2] - ref[2]) / ref[2]
    assert eo.max() < 1e-4


def test_pgd_paper_setting_k8_m64(pc, orc):
    """K=8, M=64, 10 dB targets, lambda = 1/15, learned-like per-layer eta in the clamp interval."""
    capi, precoder = pc
    H = ch.rayleigh(500, 8, 64, seed=9)
    t = ch.targets(500, 8, gamma_db=10.0)
    L = 1 / ch.paper_eta(8, 64)
    eta = np.linspace(1 / L, 1 / (2 * L), 20).astype(np.float32)
    lam = np.full(20, 1 / 15, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PGD, H, t, eta, lam)
    ref = oracle_ref(orc, 0, H, t, eta, lam)
    assert_parity(gpu, ref)


@pytest.mark.parametrize("tc", [False, True])
def test_pgd_step_normalised_on_lognormal(pc, orc, tc):
    """Per-instance eta_l / L_b with the Gershgorin bound L_b = max_k sum_j |G_kj|
    (FP32 build; split-FP16 tensor-core build, whose one global channel scale leaves
    the weak users of 8 dB log-normal gains with small FP16 rows)."""
    capi, precoder = pc
    B, K, M = 200, 8, 64
    H = ch.lognormal(B, K, M, seed=2)
    t = ch.targets(B, K)
    step = np.full(10, 0.9, np.float32)
    lam = np.full(10, 0.5, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PGD, H, t, step, lam, step_normalised=True, tensor_cores=tc)
    Wo = np.zeros_like(H, dtype=np.complex128)
    for b in range(B):
        Hb = H[b].astype(np.complex128)
        Lb = np.abs(Hb @ Hb.conj().T).sum(1).max()
        assert Lb >= orc.lambda_max(Hb) * (1 - 1e-12)
        Wo[b] = orc.ufpgd_forward(Hb, t[b], step.astype(np.float64) / Lb, lam)
    e = rel_fro(gpu[0], Wo)
    assert e.max() <= W_TOL
    # the objective ||W||_{2,1} (sum of the antenna columns' norms) of the oracle's W
    oo = np.sqrt((np.abs(Wo) ** 2).sum(axis=1)).sum(axis=1)
    assert np.max(np.abs(gpu[1] - oo) / oo) <= OBJ_TOL


# ---------------------------------------------------------------- batch mechanics

def test_empty_one_and_shared_targets(pc, orc):
    capi, precoder = pc
    plan = precoder.Plan(capi.LAYER_PROJ, 3, [(32, 4)], 64)
    mu = torch.full((3,), 0.05, device="cuda")
    H0 = torch.empty((0, 4, 32), dtype=torch.complex64, device="cuda")
    t0 = torch.ones(4, device="cuda")
    plan.solve(H0, t0, mu)  # B = 0: no-op
    H = ch.rayleigh(33, 4, 32, seed=31)
    t_shared = np.array([1.0, 2.0, 0.5, 1.5], np.float32)
    W, obj, res, fl = plan.solve(torch.from_numpy(H).cuda(), torch.from_numpy(t_shared).cuda(), mu)
    ref = oracle_ref(orc, 1, H, np.broadcast_to(t_shared, (33, 4)), [0.05] * 3)
    assert_parity((W.cpu().numpy(), obj.cpu().numpy(), res.cpu().numpy(), fl.cpu().numpy()), ref)
    W1 = plan.solve(torch.from_numpy(H[:1]).cuda(), torch.from_numpy(t_shared).cuda(), mu)[0]
    assert torch.equal(W1[0], W[0])  # per-instance result independent of the batch
    with pytest.raises(capi.PrecodeError):
        plan.solve(torch.from_numpy(ch.rayleigh(65, 4, 32, seed=1)).cuda(), t0, mu)  # B > max
    plan.close()


@pytest.mark.parametrize("M,K", [(64, 8), (256, 32), (128, 16), (64, 13)])
def test_fp16_builds_small_batches_and_shared_targets(pc, orc, M, K):
    """The split-FP16 builds (K = 8 one-warp, multi-warp exact and user-padded) on
    B = 0, 1 and 3 instances (fewer than one block's worth) with shared targets,
    T = 1 and T = 4: the oracle's results, each instance independent of the batch."""
    capi, precoder = pc
    H = ch.rician_ula(3, K, M, seed=60 + K)
    t_shared = np.linspace(0.5, 2.0, K).astype(np.float32)
    for T in (1, 4):
        mu = ch.uniform_steps(T, 0.01, 0.1, seed=61)
        plan = precoder.Plan(capi.LAYER_PROJ, T, [(M, K)], 3, tensor_cores=True)
        assert capi.precode_plan_describe(plan.handle, M, K).startswith(("solve_tch", "solve_tcwh", "solve_tg"))
        md, td = torch.from_numpy(mu).cuda(), torch.from_numpy(t_shared).cuda()
        plan.solve(torch.empty((0, K, M), dtype=torch.complex64, device="cuda"), td, md)  # no-op
        W3, o3, r3, f3 = plan.solve(torch.from_numpy(H).cuda(), td, md)
        W1 = plan.solve(torch.from_numpy(H[1:2]).cuda(), td, md)[0]
        plan.close()
        gpu = tuple(x.cpu().numpy() for x in (W3, o3, r3, f3))
        assert_parity(gpu, oracle_ref(orc, 1, H, np.broadcast_to(t_shared, (3, K)), mu))
        assert torch.equal(W1[0], W3[1])


def test_deterministic_and_host_path_identical(pc):
    capi, precoder = pc
    B = 3000
    H = ch.lognormal(B, 8, 64, seed=41)
    t = ch.targets(B, 8)
    mu = ch.fixed_workload_steps(10)
    plan = precoder.Plan(capi.LAYER_PROJ, 10, [(64, 8)], B)
    Hd, td, md = torch.from_numpy(H).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(mu).cuda()
    a = plan.solve(Hd, td, md)
    b = plan.solve(Hd, td, md)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    Hh = torch.from_numpy(H).pin_memory()
    th = torch.from_numpy(t).pin_memory()
    Wh = torch.empty_like(Hh).pin_memory()
    oh = torch.empty(B).pin_memory()
    rh = torch.empty(B).pin_memory()
    fh = torch.empty(B, dtype=torch.int32).pin_memory()
    plan.solve_host(Hh, th, torch.from_numpy(mu), None, W=Wh, obj=oh, resid=rh, flags=fh)
    assert torch.equal(Wh, a[0].cpu())
    assert torch.equal(oh, a[1].cpu()) and torch.equal(fh, a[3].cpu())
    plan.close()


@pytest.mark.parametrize("shared_t", [False, True])
def test_host_buffers_zero_copy_and_staged_identical(pc, shared_t):
    """Projected layer at K = 8, M = 64 on its split-FP16 build from host buffers:
    page-locked buffers take the zero-copy kernel (H read and W written over the
    host link from inside the kernel), pageable ones the staged copy pipeline; both
    give bitwise the device solve's outputs (B not a multiple of the chunk)."""
    capi, precoder = pc
    B = 5003
    H = ch.lognormal(B, 8, 64, seed=42)
    t = ch.targets(1, 8)[0] if shared_t else ch.targets(B, 8)
    mu = ch.fixed_workload_steps(10)
    plan = precoder.Plan(capi.LAYER_PROJ, 10, [(64, 8)], B, tensor_cores=True)
    assert capi.precode_plan_describe(plan.handle, 64, 8).startswith("solve_tch_kernel")
    a = plan.solve(torch.from_numpy(H).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(mu).cuda())
    a = [x.cpu() for x in a]
    for pinned in (True, False):
        def buf(x):
            return x.pin_memory() if pinned else x
        Hh, th = buf(torch.from_numpy(H)), buf(torch.from_numpy(np.ascontiguousarray(t)))
        Wh = buf(torch.empty(B, 8, 64, dtype=torch.complex64))
        oh, rh = buf(torch.empty(B)), buf(torch.empty(B))
        fh = buf(torch.empty(B, dtype=torch.int32))
        plan.solve_host(Hh, th, torch.from_numpy(mu), None, W=Wh, obj=oh, resid=rh, flags=fh)
        assert torch.equal(Wh, a[0]) and torch.equal(oh, a[1]), pinned
        assert torch.equal(rh, a[2]) and torch.equal(fh, a[3]), pinned
    assert plan.errors() == 0
    plan.close()


def test_fixed_workload_full_size_sampled(pc, orc):
    """The full 65,536-instance batch in the benchmark's launch configuration;
    256 sampled instances against the oracle, all flags clean, all outputs feasible."""
    capi, precoder = pc
    wl = ch.WORKLOADS["fixed"]
    H = ch.lognormal(wl.B, wl.K, wl.M, seed=wl.seed)
    t = ch.targets(wl.B, wl.K)
    mu = ch.fixed_workload_steps(wl.T)
    plan = precoder.Plan(capi.LAYER_PROJ, wl.T, [(wl.M, wl.K)], wl.B)
    W, obj, res, fl = plan.solve(torch.from_numpy(H).cuda(), torch.from_numpy(t).cuda(),
                                 torch.from_numpy(mu).cuda())
    W, obj, res, fl = W.cpu().numpy(), obj.cpu().numpy(), res.cpu().numpy(), fl.cpu().numpy()
    plan.close()
    idx = np.sort(np.random.default_rng(0).choice(wl.B, 256, replace=False))
    ref = oracle_ref(orc, 1, H[idx], t[idx], mu)
    assert_parity((W[idx], obj[idx], res[idx], fl[idx]), ref)
    assert np.all(np.isfinite(obj)) and np.all(res < 1e-4 * math.sqrt(wl.K))
    assert (fl != 0).mean() < 0.01


# ---------------------------------------------------------------- tensor-core build (K=8, M=64)

def tf32_build(tmp_path, capi, mode=None):
    """Plan options that pin K = 8, M = 64 (projected layer, or `mode`) to the
    split-TF32 build (the split-FP16 builds are that shape's defaults)."""
    mode = capi.LAYER_PROJ if mode is None else mode
    path = tmp_path / f"tune_tf32_{mode}.txt"
    path.write_text(f"{torch.cuda.get_device_name(0)}|{mode}|8|64\t"
                    "8x64/4x8/jc8/w4/b3/split/tc/exact\n")
    return dict(tensor_cores=True, autotune=True, tune_cache=str(path))


def build_kw(tmp_path, capi, build, M=64, K=8, mode=None):
    if build != "tf32":
        return dict(tensor_cores=True)
    return tf32_build(tmp_path, capi, mode) if (M, K) == (64, 8) else tcw_tf32_build(tmp_path, capi, M, K)


@pytest.mark.parametrize("mode", ["proj", "proj_tf32", "pgd", "pgd_tf32"])
def test_tensor_core_variant_parity(pc, orc, tmp_path, mode):
    """Warp-MMA builds (split FP16 by default, split TF32 pinned): same tolerances
    as the FP32 build."""
    capi, precoder = pc
    B = 1000
    kw = dict(tensor_cores=True)
    if mode == "proj_tf32":
        kw = tf32_build(tmp_path, capi)
    elif mode == "pgd_tf32":
        kw = tf32_build(tmp_path, capi, capi.LAYER_PGD)
    if mode.startswith("proj"):
        H = ch.lognormal(B, 8, 64, seed=2)
        t = ch.targets(B, 8)
        step, lam, m = ch.fixed_workload_steps(10), None, capi.LAYER_PROJ
    else:
        H = ch.rayleigh(B, 8, 64, seed=9)
        t = ch.targets(B, 8, gamma_db=10.0)
        L = 1 / ch.paper_eta(8, 64)
        step = np.linspace(1 / L, 1 / (2 * L), 20).astype(np.float32)
        lam, m = np.full(20, 1 / 15, np.float32), capi.LAYER_PGD
    plan = precoder.Plan(m, len(step), [(64, 8)], B, **kw)
    name = capi.precode_plan_describe(plan.handle, 64, 8)
    plan.close()
    assert name.startswith("solve_tc_kernel" if mode.endswith("tf32") else "solve_tch_kernel"), name
    gpu = run_gpu(precoder, m, H, t, step, lam, **kw)
    ref = oracle_ref(orc, 0 if mode.startswith("pgd") else 1, H, t, step, lam)
    e, eo = assert_parity(gpu, ref)
    if mode.startswith("proj"):
        assert np.all(gpu[2] <= 1e-4 * math.sqrt(8))


@pytest.mark.parametrize("build", ["default", "tf32"])
def test_tensor_core_variant_flags_and_uneven(pc, orc, tmp_path, build):
    capi, precoder = pc
    H = ch.rayleigh(40, 8, 64, seed=23)
    H[3, 5] = H[3, 2]   # singular
    H[7, 1, 9] = np.inf  # non-finite
    t = ch.targets(40, 8)
    mu = np.full(6, 0.05, np.float32)
    W, obj, res, fl = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, **build_kw(tmp_path, capi, build))
    assert fl[3] & capi.F_SINGULAR and not np.any(W[3]) and obj[3] == 0
    assert fl[7] & capi.F_NONFINITE
    ok = [b for b in range(40) if b not in (3, 7)]
    assert np.all(fl[ok] == 0)
    assert_parity((W[ok], obj[ok], res[ok], fl[ok]), oracle_ref(orc, 1, H[ok], t[ok], mu))


# Split-FP16 build of the projected layer (K = 8, M = 64), forced through an
# autotune cache entry naming it; each instance runs in power-of-two scaled units.
TCH_BUILDS = [3, 4]  # CTAs per SM the register budget is built for


def forced_tch(tmp_path, capi, minb):
    path = tmp_path / "tune.txt"
    path.write_text(f"{torch.cuda.get_device_name(0)}|{capi.LAYER_PROJ}|8|64\t"
                    f"8x64/4x8/jc8/w4/b{minb}/split/tc/f16/exact\n")
    return dict(tensor_cores=True, autotune=True, tune_cache=str(path))


def run_tch(capi, precoder, kw, H, t, mu, **extra):
    B = len(H)
    plan = precoder.Plan(capi.LAYER_PROJ, len(mu), [(64, 8)], max(B, 1), **kw, **extra)
    assert capi.precode_plan_describe(plan.handle, 64, 8).startswith("solve_tch_kernel")
    plan.close()
    return run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, **kw, **extra)


@pytest.mark.parametrize("minb", TCH_BUILDS)
def test_fp16_split_parity(pc, orc, tmp_path, minb):
    """Log-normal user gains (8 dB), T = 10 with the fixed workload's steps, B = 999
    (ragged last block): the FP32 tolerances against the FP64 oracle."""
    capi, precoder = pc
    kw = forced_tch(tmp_path, capi, minb)
    H = ch.lognormal(999, 8, 64, seed=41)
    t = ch.targets(999, 8)
    mu = ch.fixed_workload_steps(10)
    gpu = run_tch(capi, precoder, kw, H, t, mu)
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))
    assert np.all(gpu[2] <= 1e-4 * math.sqrt(8)) and np.all(gpu[3] == 0)


def test_fp16_split_scale_invariant(pc, orc, tmp_path):
    """Channels and targets scaled together by 1e-6 .. 1e6 per instance (W keeps its
    size, so the same mu does work everywhere): the per-instance power-of-two
    scaling keeps every instance at the same accuracy."""
    capi, precoder = pc
    kw = forced_tch(tmp_path, capi, 4)
    sc = 10.0 ** np.random.default_rng(42).uniform(-6, 6, size=128)
    H = (ch.rayleigh(128, 8, 64, seed=43) * sc[:, None, None]).astype(np.complex64)
    t = (ch.targets(128, 8) * sc[:, None]).astype(np.float32)
    mu = np.full(6, 0.05, np.float32)
    gpu = run_tch(capi, precoder, kw, H, t, mu)
    assert np.all(gpu[3] == 0)
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))


def test_fp16_split_wide_gain_spread(pc, orc, tmp_path):
    """One user 1e-5 weaker than the rest (and another 1e-3 in every other
    instance): without per-user scaling that user's channel row would sit in
    FP16's subnormals; the Gram matrix is well conditioned after equilibration, so
    the FP32 inverse is used."""
    capi, precoder = pc
    kw = forced_tch(tmp_path, capi, 4)
    H = ch.rayleigh(32, 8, 64, seed=44)
    H[:, 3] *= np.float32(1e-5)
    H[::2, 6] *= np.float32(1e-3)
    t = ch.targets(32, 8)
    mu = np.full(8, 0.02, np.float32)
    gpu = run_tch(capi, precoder, kw, H, t, mu)
    assert np.all(gpu[3] == 0)
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))


def test_fp16_split_flags_and_fp64(pc, orc, tmp_path):
    """Singular and non-finite instances and ill-conditioned ones on the FP64 path."""
    capi, precoder = pc
    kw = forced_tch(tmp_path, capi, 4)
    rs = np.random.default_rng(45)
    H = ch.rayleigh(41, 8, 64, seed=46)
    for b in range(10, 30, 2):
        H[b, 5] = H[b, 2] + (1e-3 * (rs.standard_normal(64) + 1j * rs.standard_normal(64))).astype(np.complex64)
    H[3, 5] = H[3, 2]    # singular
    H[7, 1, 9] = np.inf  # non-finite
    t = ch.targets(41, 8)
    mu = np.full(6, 0.05, np.float32)
    W, obj, res, fl = run_tch(capi, precoder, kw, H, t, mu, cond_threshold=1e3)
    assert fl[3] & capi.F_SINGULAR and not np.any(W[3]) and obj[3] == 0
    assert fl[7] & capi.F_NONFINITE
    assert np.all(fl[10:30:2] == capi.F_FP64_CHOL)
    ok = [b for b in range(41) if b not in (3, 7)]
    well = [b for b in ok if not (10 <= b < 30 and b % 2 == 0)]
    assert np.all(fl[well] == 0)
    gpu, ref = (W[ok], obj[ok], res[ok], fl[ok]), oracle_ref(orc, 1, H[ok], t[ok], mu)
    sel = np.isin(ok, well)
    assert_parity(tuple(x[sel] for x in gpu), tuple(x[sel] for x in ref))
    assert_parity(gpu, ref)


def test_fp16_split_full_size_sampled(pc, orc, tmp_path):
    capi, precoder = pc
    wl = ch.WORKLOADS["fixed"]
    kw = forced_tch(tmp_path, capi, 4)
    H = ch.lognormal(wl.B, wl.K, wl.M, seed=wl.seed)
    t = ch.targets(wl.B, wl.K)
    mu = ch.fixed_workload_steps(wl.T)
    plan = precoder.Plan(capi.LAYER_PROJ, wl.T, [(wl.M, wl.K)], wl.B, **kw)
    assert capi.precode_plan_describe(plan.handle, wl.M, wl.K).startswith("solve_tch_kernel")
    W, obj, res, fl = plan.solve(torch.from_numpy(H).cuda(), torch.from_numpy(t).cuda(),
                                 torch.from_numpy(mu).cuda())
    W, obj, res, fl = W.cpu().numpy(), obj.cpu().numpy(), res.cpu().numpy(), fl.cpu().numpy()
    plan.close()
    idx = np.sort(np.random.default_rng(3).choice(wl.B, 256, replace=False))
    assert_parity((W[idx], obj[idx], res[idx], fl[idx]), oracle_ref(orc, 1, H[idx], t[idx], mu))
    assert np.all(res < 1e-4 * math.sqrt(wl.K)) and (fl != 0).mean() < 0.01


# Multi-warp split-FP16 builds (projected layer; exact bucket shapes and user-padded
# builds), forced through an autotune cache entry naming the build.
TCWH_BUILDS = [  # (M, K, KW, CTAs per SM, exact)
    (256, 32, 4, 2, True), (128, 16, 2, 6, True), (256, 27, 4, 2, False), (128, 11, 2, 6, False),
    (64, 29, 4, 4, False), (64, 13, 2, 8, False)]


def forced_tcwh(tmp_path, capi, M, K, kw, minb, exact):
    path = tmp_path / "tune_tcwh.txt"
    key = f"{8 * kw}x{M}/{kw}x8/jc8/w{kw}/b{minb}/split/tc/f16/{'exact' if exact else 'generic'}"
    path.write_text(f"{torch.cuda.get_device_name(0)}|{capi.LAYER_PROJ}|{K}|{M}\t{key}\n")
    return dict(tensor_cores=True, autotune=True, tune_cache=str(path))


def run_tcwh(capi, precoder, kw, H, t, mu, **extra):
    B, K, M = H.shape
    plan = precoder.Plan(capi.LAYER_PROJ, len(mu), [(M, K)], max(B, 1), **kw, **extra)
    assert capi.precode_plan_describe(plan.handle, M, K).startswith("solve_tcwh_kernel")
    plan.close()
    return run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, **kw, **extra)


@pytest.mark.parametrize("M,K,kw,minb,exact", TCWH_BUILDS)
def test_fp16_multiwarp_parity(pc, orc, tmp_path, M, K, kw, minb, exact):
    """Rician channels (K-factor 0-10 dB, ULA), T = 10 uniform steps: the FP32
    tolerances against the FP64 oracle, exact and user-padded builds."""
    capi, precoder = pc
    B = 300 if M == 256 else 600
    H = ch.rician_ula(B, K, M, seed=50 + K)
    t = ch.targets(B, K)
    mu = ch.uniform_steps(10, 0.01, 0.1, seed=51)
    gpu = run_tcwh(capi, precoder, forced_tcwh(tmp_path, capi, M, K, kw, minb, exact), H, t, mu)
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))
    assert np.all(gpu[2] <= 1e-4 * math.sqrt(K))


def test_fp16_multiwarp_scales_and_gain_spread(pc, orc, tmp_path):
    """Channels and targets over 1e-5 .. 1e5 together per instance, and one user
    1e-4 weaker than the rest in every other instance."""
    capi, precoder = pc
    M, K = 128, 16
    kw = forced_tcwh(tmp_path, capi, M, K, 2, 6, True)
    sc = 10.0 ** np.random.default_rng(52).uniform(-5, 5, size=200)
    H = (ch.rayleigh(200, K, M, seed=53) * sc[:, None, None]).astype(np.complex64)
    H[::2, 5] *= np.float32(1e-4)
    t = (ch.targets(200, K) * sc[:, None]).astype(np.float32)
    mu = np.full(8, 0.03, np.float32)
    gpu = run_tcwh(capi, precoder, kw, H, t, mu)
    assert np.all(gpu[3] == 0)
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_fp16_multiwarp_flags_and_fp64(pc, orc, tmp_path, eps):
    """Singular and non-finite instances and ill-conditioned ones on the FP64 path
    (near-collinear user pairs eps apart: F' = E' G'^{-T} grows with the condition,
    and the per-warp range check moves powers of two onto the channel operand or,
    at eps = 1e-4 (condition ~1e8), runs those layers' update as split TF32)."""
    capi, precoder = pc
    M, K = 256, 32
    kw = forced_tcwh(tmp_path, capi, M, K, 4, 2, True)
    rs = np.random.default_rng(54)
    H = ch.rayleigh(24, K, M, seed=55)
    for b in range(8, 20, 2):
        H[b, 9] = H[b, 4] + (eps * (rs.standard_normal(M) + 1j * rs.standard_normal(M))).astype(np.complex64)
    H[3, 7] = H[3, 2]    # singular
    H[5, 1, 9] = np.inf  # non-finite
    t = ch.targets(24, K)
    mu = np.full(6, 0.05, np.float32)
    W, obj, res, fl = run_tcwh(capi, precoder, kw, H, t, mu, cond_threshold=1e3)
    assert fl[3] & capi.F_SINGULAR and not np.any(W[3]) and obj[3] == 0
    assert fl[5] & capi.F_NONFINITE
    assert np.all(fl[8:20:2] == capi.F_FP64_CHOL)
    ok = [b for b in range(24) if b not in (3, 5)]
    well = [b for b in ok if not (8 <= b < 20 and b % 2 == 0)]
    assert np.all(fl[well] == 0)
    gpu, ref = (W[ok], obj[ok], res[ok], fl[ok]), oracle_ref(orc, 1, H[ok], t[ok], mu)
    sel = np.isin(ok, well)
    assert_parity(tuple(x[sel] for x in gpu), tuple(x[sel] for x in ref))
    assert np.all(np.isfinite(W[ok])) and np.all(np.isfinite(obj[ok]))
    assert_parity(gpu, ref)


# The tcgen05 builds (any K <= 32 users at M = 256: operands in shared memory,
# accumulators in tensor memory), forced through an autotune cache entry: the row
# build (a warp per 16 rows of W) and the transposed one (a thread per antenna,
# Q^T in tensor memory).
TG_KEY = "32x256/4x8/jc8/w8/b1/split/tc/f16/tg/generic"
TG_KEYS = {"tg": TG_KEY, "tgt": "32x256/4x8/jc8/w8/b1/split/tc/f16/tg/tgt/generic"}
TG_NAMES = {"tg": "solve_tg_kernel<1>", "tgt": "solve_tgt_kernel<1>"}


@pytest.fixture(params=["tg", "tgt"])
def tgb(request):
    return request.param


def forced_tg(tmp_path, capi, K, M=256, build="tg"):
    path = tmp_path / f"tune_{build}.txt"
    path.write_text(f"{torch.cuda.get_device_name(0)}|{capi.LAYER_PROJ}|{K}|{M}\t{TG_KEYS[build]}\n")
    return dict(tensor_cores=True, autotune=True, tune_cache=str(path))


def run_tg(capi, precoder, tmp_path, H, t, mu, build="tg", **extra):
    B, K, M = H.shape
    kw = forced_tg(tmp_path, capi, K, M, build)
    plan = precoder.Plan(capi.LAYER_PROJ, len(mu), [(M, K)], max(B, 1), **kw, **extra)
    assert capi.precode_plan_describe(plan.handle, M, K) == TG_NAMES[build]
    plan.close()
    return run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, **kw, **extra)


@pytest.mark.parametrize("K,B", [(32, 400), (28, 300), (25, 170)])
def test_tcgen05_parity(pc, orc, tmp_path, K, B, tgb):
    """Rician ULA channels (K-factor 0-10 dB), T = 10 uniform steps: the FP32 bar
    per instance against the FP64 oracle, with more instances than one round of
    the persistent CTAs (one per SM) and users padded to 32."""
    capi, precoder = pc
    H = ch.rician_ula(B, K, 256, seed=60 + K)
    t = ch.targets(B, K)
    mu = ch.uniform_steps(10, 0.01, 0.1, seed=61)
    gpu = run_tg(capi, precoder, tmp_path, H, t, mu, tgb)
    assert np.all(gpu[3] == 0)
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))
    assert np.all(gpu[2] <= 1e-4 * math.sqrt(K))


@pytest.mark.parametrize("T", [1, 40])
def test_tcgen05_layer_counts(pc, orc, tmp_path, T, tgb):
    """One layer (the minimum-norm start W^(0) and a single shrink and
    projection) and 40 layers, on log-normal Rayleigh channels."""
    capi, precoder = pc
    H = ch.lognormal(160, 32, 256, seed=62)
    t = ch.targets(160, 32)
    mu = ch.uniform_steps(T, 0.01, 0.1, seed=63)
    gpu = run_tg(capi, precoder, tmp_path, H, t, mu, tgb)
    assert np.all(gpu[3] == 0)
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))


def test_tcgen05_scales_and_gain_spread(pc, orc, tmp_path, tgb):
    """Channels and targets over 1e-5 .. 1e5 together per instance, and one user
    1e-4 weaker than the rest in every other instance."""
    capi, precoder = pc
    K = 32
    sc = 10.0 ** np.random.default_rng(64).uniform(-5, 5, size=160)
    H = (ch.rayleigh(160, K, 256, seed=65) * sc[:, None, None]).astype(np.complex64)
    H[::2, 5] *= np.float32(1e-4)
    t = (ch.targets(160, K) * sc[:, None]).astype(np.float32)
    mu = np.full(8, 0.03, np.float32)
    gpu = run_tg(capi, precoder, tmp_path, H, t, mu, tgb)
    assert np.all(gpu[3] == 0)
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))


@pytest.mark.parametrize("eps", [1e-3, 1e-4])
def test_tcgen05_flags_and_fp64(pc, orc, tmp_path, eps, tgb):
    """A singular Gram matrix, a non-finite input and near-collinear user pairs eps
    apart (the FP64 orthonormal-basis path, its layers on the tensor cores), with
    the per-row range scale of F; the FP32 bar on every solved instance."""
    capi, precoder = pc
    M, K = 256, 32
    rs = np.random.default_rng(66)
    H = ch.rayleigh(24, K, M, seed=67)
    for b in range(8, 20, 2):
        H[b, 9] = H[b, 4] + (eps * (rs.standard_normal(M) + 1j * rs.standard_normal(M))).astype(np.complex64)
    H[3, 7] = H[3, 2]    # singular
    H[5, 1, 9] = np.inf  # non-finite
    t = ch.targets(24, K)
    mu = np.full(6, 0.05, np.float32)
    W, obj, res, fl = run_tg(capi, precoder, tmp_path, H, t, mu, tgb, cond_threshold=1e3)
    assert fl[3] & capi.F_SINGULAR and not np.any(W[3]) and obj[3] == 0
    assert fl[5] & capi.F_NONFINITE
    assert np.all(fl[8:20:2] == capi.F_FP64_CHOL)
    ok = [b for b in range(24) if b not in (3, 5)]
    well = [b for b in ok if not (8 <= b < 20 and b % 2 == 0)]
    assert np.all(fl[well] == 0)
    assert_parity((W[ok], obj[ok], res[ok], fl[ok]), oracle_ref(orc, 1, H[ok], t[ok], mu))


def test_tcgen05_deterministic(pc, tmp_path, tgb):
    """Bitwise the same output on a second call and inside a larger batch."""
    capi, precoder = pc
    H = ch.rician_ula(200, 32, 256, seed=68)
    t = ch.targets(200, 32)
    mu = ch.uniform_steps(10, 0.01, 0.1, seed=69)
    a = run_tg(capi, precoder, tmp_path, H, t, mu, tgb)
    b = run_tg(capi, precoder, tmp_path, H, t, mu, tgb)
    c = run_tg(capi, precoder, tmp_path, H[:37], t[:37], mu, tgb)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    for x, y in zip(a, c):
        assert np.array_equal(x[:37], y)


@pytest.mark.parametrize("build", ["default", "tf32"])
def test_tensor_core_ill_conditioned_uses_fp64(pc, orc, tmp_path, build):
    """K = 8, M = 64 with one almost collinear user pair in every other instance:
    the tensor-core kernel's register Gauss-Jordan flags the pivot spread and the
    FP64 setup forms Q instead; the rest keep the FP32 inverse and MMA-formed Q."""
    capi, precoder = pc
    rs = np.random.default_rng(6)
    H = ch.rayleigh(16, 8, 64, seed=24)
    for b in range(0, 16, 2):
        H[b, 5] = H[b, 2] + (1e-3 * (rs.standard_normal(64) + 1j * rs.standard_normal(64))).astype(np.complex64)
    t = ch.targets(16, 8)
    mu = np.full(4, 0.02, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, cond_threshold=1e3,
                  **build_kw(tmp_path, capi, build))
    assert np.all(gpu[3][0::2] == capi.F_FP64_CHOL)
    assert np.all(gpu[3][1::2] == 0)
    ref = oracle_ref(orc, 1, H, t, mu)
    assert_parity(tuple(x[1::2] for x in gpu), tuple(x[1::2] for x in ref))
    assert_parity(gpu, ref)


def tcw_tf32_build(tmp_path, capi, M, K, exact=True):
    """Plan options that pin a multi-warp bucket of the projected layer to its
    split-TF32 build (the split-FP16 build is the default there)."""
    kw = -(-K // 8)
    minb = {64: {1: 16, 2: 8, 3: 5, 4: 4}, 128: {1: 12, 2: 6, 3: 4, 4: 3},
            256: {1: 8, 2: 4, 3: 2, 4: 2}}[M][kw]
    path = tmp_path / "tune_tcw32.txt"
    path.write_text(f"{torch.cuda.get_device_name(0)}|{capi.LAYER_PROJ}|{K}|{M}\t"
                    f"{8 * kw}x{M}/{kw}x8/jc8/w{kw}/b{minb}/split/tc/{'exact' if exact else 'generic'}\n")
    return dict(tensor_cores=True, autotune=True, tune_cache=str(path))


@pytest.mark.parametrize("K,M,B", [(16, 128, 2600), (32, 256, 700)])
@pytest.mark.parametrize("mode", ["proj", "proj_tf32", "pgd"])
def test_tensor_core_large_buckets(pc, orc, tmp_path, K, M, B, mode):
    """Multi-warp tensor-core builds (one CTA per instance; for the projected layer
    split FP16 by default, tcgen05 at 32 x 256, split TF32 pinned; split TF32 for
    the paper layer) against the oracle, over more instances than one persistent
    round, so CTAs take a ragged number of instances."""
    capi, precoder = pc
    kw = tcw_tf32_build(tmp_path, capi, M, K) if mode == "proj_tf32" else dict(tensor_cores=True)
    if mode.startswith("proj"):
        H = ch.rician_ula(B, K, M, seed=5)
        t = ch.targets(B, K)
        step, lam, m = ch.uniform_steps(10, 0.01, 0.1, seed=7), None, capi.LAYER_PROJ
    else:
        H = ch.rayleigh(B, K, M, seed=9)
        t = ch.targets(B, K, gamma_db=10.0)
        L = 1 / ch.paper_eta(K, M)
        step = np.linspace(1 / L, 1 / (2 * L), 10).astype(np.float32)
        lam, m = np.full(10, 1 / 15, np.float32), capi.LAYER_PGD
    plan = precoder.Plan(m, len(step), [(M, K)], B, **kw)
    name = capi.precode_plan_describe(plan.handle, M, K)
    plan.close()
    expect = {"proj": "solve_tgt_kernel" if M == 256 else "solve_tcwh_kernel"}.get(mode, "solve_tcw_kernel")
    assert name.startswith(expect), name
    gpu = run_gpu(precoder, m, H, t, step, lam, **kw)
    ref = oracle_ref(orc, 0 if mode == "pgd" else 1, H, t, step, lam)
    assert_parity(gpu, ref)


@pytest.mark.parametrize("K,M,build", [(5, 64, "default"), (13, 64, "default"), (27, 64, "default"),
                                       (3, 128, "default"), (20, 128, "default"), (9, 256, "default"),
                                       (27, 256, "default"), (13, 64, "tf32"), (20, 128, "tf32"),
                                       (27, 256, "tf32")])
def test_tensor_core_padded_users(pc, orc, tmp_path, K, M, build):
    """User-padded tensor-core builds (K < KB users at exactly MB antennas): the
    padded rows stay zero and the real users match the oracle."""
    capi, precoder = pc
    B = 200
    H = ch.rician_ula(B, K, M, seed=30 + K)
    t = ch.targets(B, K)
    mu = ch.uniform_steps(10, 0.01, 0.1, seed=7)
    kw = tcw_tf32_build(tmp_path, capi, M, K, exact=False) if build == "tf32" else dict(tensor_cores=True)
    plan = precoder.Plan(capi.LAYER_PROJ, 10, [(M, K)], B, **kw)
    name = capi.precode_plan_describe(plan.handle, M, K)
    plan.close()
    # K <= 8 has only split-TF32 padded builds (one warp); 9..32 default to split FP16,
    # 25..32 at 256 antennas to the transposed tcgen05 build
    expect = "solve_tcw_kernel"
    if build == "default" and K > 8:
        expect = "solve_tgt_kernel" if (M == 256 and K > 24) else "solve_tcwh_kernel"
    assert name.startswith(expect), name
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, **kw)
    ref = oracle_ref(orc, 1, H, t, mu)
    ok = gpu[3] == 0
    assert ok.sum() > B // 2
    assert_parity(tuple(x[ok] for x in gpu), tuple(x[ok] for x in ref))
    if np.any(~ok):  # FP64-path instances (orthonormal basis): the same bar
        assert np.all(gpu[3][~ok] == capi.F_FP64_CHOL)
        assert_parity(tuple(x[~ok] for x in gpu), tuple(x[~ok] for x in ref))


@pytest.mark.parametrize("build", ["default", "tf32"])
def test_tensor_core_large_flags_and_fp64(pc, orc, tmp_path, build):
    """32 x 256 on the multi-warp builds: a singular Gram matrix, a non-finite
    input and near-collinear user pairs (FP64 Gauss-Jordan path)."""
    capi, precoder = pc
    rs = np.random.default_rng(8)
    H = ch.rayleigh(24, 32, 256, seed=25)
    H[3, 7] = H[3, 2]
    H[5, 0, 9] = np.nan
    for b in range(8, 24, 2):
        H[b, 20] = H[b, 11] + (1e-3 * (rs.standard_normal(256) + 1j * rs.standard_normal(256))).astype(np.complex64)
    t = ch.targets(24, 32)
    mu = np.full(4, 0.02, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, cond_threshold=1e3,
                  **build_kw(tmp_path, capi, build, 256, 32))
    W, obj, res, fl = gpu
    assert fl[3] & capi.F_SINGULAR and fl[3] & capi.F_FP64_CHOL and not np.any(W[3])
    assert fl[5] & capi.F_NONFINITE
    fb = list(range(8, 24, 2))
    assert np.all(fl[fb] == capi.F_FP64_CHOL)
    ok = [b for b in range(24) if b not in (3, 5) and b not in fb]
    assert np.all(fl[ok] == 0)
    assert_parity(tuple(x[ok] for x in gpu), oracle_ref(orc, 1, H[ok], t[ok], mu))
    assert_parity(tuple(x[fb] for x in gpu), oracle_ref(orc, 1, H[fb], t[fb], mu))


def test_tensor_core_kernels_independent_of_earlier_kernels(pc, tmp_path):
    """Each tensor-core solve kernel gives bitwise the same output fresh and after
    other kernels (with other shared-memory layouts) ran on the device: every
    shared-memory operand is written before it is read."""
    capi, precoder = pc
    cases = [(capi.LAYER_PROJ, 8, 64, "default"), (capi.LAYER_PROJ, 8, 64, "tf32"),
             (capi.LAYER_PGD, 8, 64, "default"), (capi.LAYER_PGD, 8, 64, "tf32"),
             (capi.LAYER_PROJ, 16, 128, "default"),
             (capi.LAYER_PROJ, 32, 256, "default"), (capi.LAYER_PROJ, 32, 256, "tf32"),
             (capi.LAYER_PROJ, 13, 64, "default")]
    runs = {}
    for rep in range(2):
        for mode, K, M, build in (cases if rep == 0 else cases[::-1]):
            H = ch.rician_ula(600, K, M, seed=70 + K)
            t = ch.targets(600, K)
            step = ch.uniform_steps(6, 0.01, 0.1, seed=7) if mode == capi.LAYER_PROJ else \
                np.full(6, ch.paper_eta(K, M), np.float32)
            lam = None if mode == capi.LAYER_PROJ else np.full(6, 1 / 15, np.float32)
            out = run_gpu(precoder, mode, H, t, step, lam, **build_kw(tmp_path, capi, build, M, K, mode))
            if rep == 0:
                runs[(mode, K, M, build)] = out
            else:
                for a, b in zip(out, runs[(mode, K, M, build)]):
                    assert np.array_equal(a, b), (mode, K, M, build)


def test_tensor_core_full_size_sampled(pc, orc, tmp_path):
    """The split-TF32 build on the full fixed workload (the split-FP16 build has its
    own full-size test)."""
    capi, precoder = pc
    wl = ch.WORKLOADS["fixed"]
    H = ch.lognormal(wl.B, wl.K, wl.M, seed=wl.seed)
    t = ch.targets(wl.B, wl.K)
    mu = ch.fixed_workload_steps(wl.T)
    plan = precoder.Plan(capi.LAYER_PROJ, wl.T, [(wl.M, wl.K)], wl.B, **tf32_build(tmp_path, capi))
    assert "solve_tc_kernel" in capi.precode_plan_describe(plan.handle, wl.M, wl.K)
    W, obj, res, fl = plan.solve(torch.from_numpy(H).cuda(), torch.from_numpy(t).cuda(),
                                 torch.from_numpy(mu).cuda())
    W, obj, res, fl = W.cpu().numpy(), obj.cpu().numpy(), res.cpu().numpy(), fl.cpu().numpy()
    plan.close()
    idx = np.sort(np.random.default_rng(1).choice(wl.B, 256, replace=False))
    assert_parity((W[idx], obj[idx], res[idx], fl[idx]), oracle_ref(orc, 1, H[idx], t[idx], mu))
    assert np.all(res < 1e-4 * math.sqrt(wl.K)) and (fl != 0).mean() < 0.01


# ---------------------------------------------------------------- conditioning sweep

def cond_hat(H):
    """Pivot ratio max d / min d of the LDL^H factorisation of the equilibrated
    Gram matrix D H H^H D, D = diag(H H^H)^{-1/2} (FP64 numpy): the condition
    estimate the kernels compare with the threshold of the FP64 path."""
    out = []
    for Hb in H.astype(np.complex128):
        G = Hb @ Hb.conj().T
        d = 1 / np.sqrt(np.real(np.diag(G)))
        p = np.real(np.diag(np.linalg.cholesky(d[:, None] * G * d[None, :]))) ** 2
        out.append(p.max() / p.min())
    return np.array(out)


def near_collinear(B, K, M, eps, seed):
    """CN(0,1) channels where, per instance, one user's row is another user's
    row plus eps times CN(0,1) noise (equilibrated Gram condition ~ 1 / eps^2)."""
    rs = np.random.default_rng(seed + 7)
    H = ch.rayleigh(B, K, M, seed=seed).copy()
    for b in range(B):
        i, j = rs.choice(K, 2, replace=False)
        H[b, j] = H[b, i] + (eps * (rs.standard_normal(M) + 1j * rs.standard_normal(M))).astype(np.complex64)
    return H


COND_SWEEP = [  # (build label, K, M): every kernel family of the projected layer
    ("ffma", 4, 32), ("ffma", 11, 100), ("default", 8, 64), ("tf32", 8, 64),
    ("default", 16, 128), ("default", 32, 256), ("tf32", 32, 256), ("default", 27, 256)]


@pytest.mark.parametrize("build,K,M", COND_SWEEP)
def test_fp64_path_conditioning_sweep(pc, orc, tmp_path, build, K, M):
    """Rician ULA channels (estimates ~2 to ~8: the FP32 setup) and near-collinear
    user pairs eps apart, eps from 1e-1 to 1e-5 (equilibrated Gram condition
    estimates from ~50 to ~5e9: the FP64 path, whose layers run in an orthonormal
    basis of the channel's row space), default threshold (16), T = 20: every
    instance meets the 1e-4 / 1e-5 bar; FP64_CHOL is set exactly on the instances
    whose estimate is clearly above the threshold."""
    capi, precoder = pc
    per = 6 if M >= 128 else 12
    H = np.concatenate([ch.rician_ula(per, K, M, seed=190 + K)] +
                       [near_collinear(per, K, M, eps, seed=200 + K + i)
                        for i, eps in enumerate((1e-1, 1e-2, 1e-3, 1e-4, 1e-5))])
    t = ch.targets(len(H), K)
    mu = np.full(20, 0.03, np.float32)
    if build == "ffma":
        kw = {}
    elif build == "tf32":
        kw = build_kw(tmp_path, capi, "tf32", M, K)
    else:
        kw = dict(tensor_cores=True)
    gpu = run_gpu(precoder, capi.LAYER_PROJ, H, t, mu, **kw)
    kap = cond_hat(H)
    fl = gpu[3]
    assert np.all(fl[kap > 32] == capi.F_FP64_CHOL) and np.all(fl[kap < 8] == 0), (kap, fl)
    assert (fl == 0).sum() >= per // 2 and (fl != 0).sum() >= 4 * per
    assert_parity(gpu, oracle_ref(orc, 1, H, t, mu))
    assert np.all(np.isfinite(gpu[0]))


# ---------------------------------------------------------------- classical PGD, 5,000 layers

@pytest.mark.parametrize("tc", [False, True])
def test_pgd_5000_layers_paper_setting(pc, orc, tc):
    """The classical PGD of Sec. VI-C through the paper-layer kernels: 5,000
    layers with the constant step eta = 1/L~ and lambda = 1/15, K = 8, M = 64,
    CN(0,1) channels, gamma = 10 dB.  After 5,000 layers W and the objective still
    meet the 1e-4 / 1e-5 bar against the FP64 oracle (the tensor-core build adds
    each update to W with a rounded FP32 add, so the MMA accumulation's rounding
    does not accumulate into a drift)."""
    capi, precoder = pc
    B, K, M, T = 32, 8, 64, 5000
    H = ch.rayleigh(B, K, M, seed=500)
    t = ch.targets(B, K, gamma_db=10.0)
    eta = np.full(T, ch.paper_eta(K, M), np.float32)
    lam = np.full(T, 1 / 15, np.float32)
    gpu = run_gpu(precoder, capi.LAYER_PGD, H, t, eta, lam, tensor_cores=tc)
    ref = oracle_ref(orc, 0, H, t, eta, lam)
    assert_parity(gpu, ref)
