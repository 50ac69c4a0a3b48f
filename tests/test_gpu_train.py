"""Adjoint (training) kernels on the GPU against the FP64 oracle's reverse mode.

The oracle's gradients are themselves pinned to central finite differences
(tests/test_oracle_pins.py).  Instances with a column within reach of a shrink
kink (|r - tau| small on some layer) are left out, as there the FP32 and FP64
forward passes may sit on different sides of the kink.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2304_12745_gb300 import channels as ch

pytestmark = pytest.mark.gpu


def _far_from_kinks_proj(orc, H, t, mu, margin):
    keep = []
    for b in range(len(H)):
        _, _, tr = orc.ufproj_forward(H[b], t[b], mu, trace=True)
        d = min(np.abs(np.linalg.norm(tr[l], axis=0) - mu[l]).min() for l in range(len(mu)))
        keep.append(d > margin)
    return np.array(keep)


def _far_from_kinks_pgd(orc, H, t, eta, lam, margin):
    keep = []
    for b in range(len(H)):
        _, tr = orc.ufpgd_forward(H[b], t[b], eta, lam, trace=True)
        d = np.inf
        for l in range(len(eta)):
            V = tr[l] - eta[l] * ((tr[l] @ H[b].T - np.diag(t[b])) @ H[b].conj())
            d = min(d, np.abs(np.linalg.norm(V, axis=0) - lam[l] * eta[l]).min())
        keep.append(d > margin)
    return np.array(keep)


def _train_step(plan, H, t, step, lam, a):
    from paper_2304_12745_gb300 import capi
    B, K, M = H.shape
    Hd = torch.from_numpy(H.astype(np.complex64)).cuda()
    td = torch.from_numpy(np.ascontiguousarray(t, np.float32)).cuda()
    sd = torch.tensor(step, dtype=torch.float32, device="cuda")
    ld = torch.tensor(lam, dtype=torch.float32, device="cuda") if lam is not None else None
    loss = torch.empty(1, device="cuda")
    ds = torch.empty(len(step), device="cuda")
    dl = torch.empty(len(step), device="cuda") if lam is not None else None
    capi.precode_train_step(plan.handle, M, K, B, Hd, td, K, sd, ld, a, loss, ds, dl, None,
                            torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return (float(loss.item()), ds.cpu().numpy().astype(np.float64),
            None if dl is None else dl.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("K,M,T,tc", [(4, 32, 6, False), (8, 64, 10, False), (8, 64, 10, True),
                                      (8, 64, 10, "tf32")])
def test_projected_gradient_matches_oracle(orc, monkeypatch, K, M, T, tc):
    """FP32 build, and the tensor-core builds of the forward + adjoint pass (split
    FP16 by default; split TF32 with PRECODE_TRAIN_TF32)."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan
    if tc == "tf32":
        monkeypatch.setenv("PRECODE_TRAIN_TF32", "1")
    B0 = 64
    H = ch.rayleigh(B0, K, M, seed=40 + K).astype(np.complex128)
    H = H.astype(np.complex64).astype(np.complex128)  # the GPU sees complex64
    t = np.ones((B0, K))
    mu = ch.uniform_steps(T, 0.02, 0.08, seed=41).astype(np.float32).astype(np.float64)
    keep = _far_from_kinks_proj(orc, H, t, mu, 2e-5)
    H, t = H[keep], t[keep]
    B = len(H)
    assert B >= 16
    a = 1.0
    ref = [orc.ufproj_grad(H[b], t[b], mu, a) for b in range(B)]
    loss_o = np.mean([r[0] for r in ref])
    g_o = np.mean([r[1] for r in ref], axis=0)
    plan = Plan(capi.LAYER_PROJ, T, [(M, K)], B, tensor_cores=bool(tc))
    loss, g, _ = _train_step(plan, H, t, mu, None, a)
    plan.close()
    assert loss == pytest.approx(loss_o, rel=1e-5)
    assert np.allclose(g, g_o, rtol=1e-3, atol=1e-3 * np.abs(g_o).max()), (g, g_o)


@pytest.mark.parametrize("K,M,tc", [(4, 32, False), (8, 64, True)])
def test_paper_layer_gradient_matches_oracle(orc, K, M, tc):
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan
    T, B0 = 5, 64
    H = ch.rayleigh(B0, K, M, seed=50).astype(np.complex128)
    t = np.ones((B0, K))
    eta0 = ch.paper_eta(K, M)
    rs = np.random.default_rng(51)
    eta = (eta0 * rs.uniform(0.5, 1.0, T)).astype(np.float32).astype(np.float64)
    lam = rs.uniform(0.5, 3.0, T).astype(np.float32).astype(np.float64)
    keep = _far_from_kinks_pgd(orc, H, t, eta, lam, 2e-5)
    H, t = H[keep], t[keep]
    B = len(H)
    assert B >= 16
    a = 1 / 15
    ref = [orc.ufpgd_grad(H[b], t[b], eta, lam, a) for b in range(B)]
    loss_o = np.mean([r[0] for r in ref])
    ge_o = np.mean([r[1] for r in ref], axis=0)
    gl_o = np.mean([r[2] for r in ref], axis=0)
    plan = Plan(capi.LAYER_PGD, T, [(M, K)], B, tensor_cores=tc)
    loss, ge, gl = _train_step(plan, H, t, eta, lam, a)
    plan.close()
    assert loss == pytest.approx(loss_o, rel=1e-5)
    assert np.allclose(ge, ge_o, rtol=1e-3, atol=1e-3 * np.abs(ge_o).max()), (ge, ge_o)
    assert np.allclose(gl, gl_o, rtol=1e-3, atol=1e-3 * np.abs(gl_o).max()), (gl, gl_o)


@pytest.mark.parametrize("tc", [False, True, "tf32"])
def test_gradient_matches_central_differences_of_the_gpu_loss(monkeypatch, tc):
    """Central differences (h = 1e-3) of the GPU's own FP32 batch loss."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan
    if tc == "tf32":
        monkeypatch.setenv("PRECODE_TRAIN_TF32", "1")
    K, M, T, B = 8, 64, 10, 2048
    H = ch.rayleigh(B, K, M, seed=60)
    t = np.ones((B, K), np.float32)
    mu = ch.uniform_steps(T, 0.02, 0.08, seed=61).astype(np.float64)
    plan = Plan(capi.LAYER_PROJ, T, [(M, K)], B, tensor_cores=bool(tc))
    _, g, _ = _train_step(plan, H, t, mu, None, 1.0)
    h = 1e-3
    for l in (0, 4, 9):
        mp, mm = mu.copy(), mu.copy()
        mp[l] += h
        mm[l] -= h
        fd = (_train_step(plan, H, t, mp, None, 1.0)[0] - _train_step(plan, H, t, mm, None, 1.0)[0]) / (2 * h)
        assert fd == pytest.approx(g[l], rel=2e-2, abs=2e-2 * np.abs(g).max()), (l, fd, g[l])
    plan.close()


def test_tensor_core_training_independent_of_earlier_kernels():
    """The projected-layer training kernel after paper-layer kernels (which leave
    their own data in shared memory) gives the same finite gradient as alone:
    every shared-memory operand is written before it is read."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan
    K, M, T, B = 8, 64, 20, 4096
    H = ch.rayleigh(B, K, M, seed=62)
    t = np.full((B, K), math.sqrt(10.0), np.float32)
    mu = np.full(T, 0.05)
    plan = Plan(capi.LAYER_PROJ, T, [(M, K)], B, tensor_cores=True)
    alone = _train_step(plan, H, t, mu, None, 1.0)
    for tc in (True, False):
        pg = Plan(capi.LAYER_PGD, T, [(M, K)], B, tensor_cores=tc)
        _train_step(pg, H, t, np.full(T, ch.paper_eta(K, M)), np.full(T, 0.07), 1.0)
        pg.close()
        after = _train_step(plan, H, t, mu, None, 1.0)
        assert np.all(np.isfinite(after[1]))
        assert after[0] == alone[0] and np.array_equal(after[1], alone[1])
    plan.close()


def test_train_step_deterministic_and_trainer_resume():
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.training import UnfoldedTrainer
    K, M, T, Bt = 8, 64, 10, 512
    tr = UnfoldedTrainer(capi.LAYER_PROJ, T, K, M, Bt, a=1.0, lr=2e-3)
    t = torch.ones(K, device="cuda")
    H0 = tr.make_batch(0, seed=4)
    l1 = tr.loss(H0, t)
    l2 = tr.loss(H0, t)
    assert float(l1) == float(l2)
    losses = [tr.train_step(tr.make_batch(i, seed=4), t) for i in range(8)]
    ref = tr.step.detach().clone()
    # resume: 4 steps, save, new trainer, load, 4 more
    a = UnfoldedTrainer(capi.LAYER_PROJ, T, K, M, Bt, a=1.0, lr=2e-3)
    for i in range(4):
        a.train_step(a.make_batch(i, seed=4), t)
    state = a.state_dict()
    b = UnfoldedTrainer(capi.LAYER_PROJ, T, K, M, Bt, a=1.0, lr=2e-3)
    b.load_state_dict(state)
    for i in range(4, 8):
        b.train_step(b.make_batch(i, seed=4), t)
    assert torch.equal(b.step.detach(), ref)
    assert np.all(np.isfinite(losses))


def test_paper_layer_training_reduces_the_cost():
    """Adam on eta, lambda with the paper's projections lowers the unsupervised cost."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.training import UnfoldedTrainer, mp_bound
    K, M, T, Bt = 8, 64, 10, 1024
    tr = UnfoldedTrainer(capi.LAYER_PGD, T, K, M, Bt, a=1 / 15, lr=1e-3)
    t = torch.full((K,), math.sqrt(10.0), device="cuda")
    Hv = tr.make_batch(999, seed=5)
    before = float(tr.loss(Hv, t))
    for i in range(40):
        tr.train_step(tr.make_batch(i, seed=5), t)
    after = float(tr.loss(Hv, t))
    assert after < before
    L = mp_bound(K, M)
    assert torch.all(tr.step >= 1 / (2 * L) - 1e-9) and torch.all(tr.step <= 1 / L + 1e-9)
    assert torch.all(tr.lam >= 0)


@pytest.mark.parametrize("mode", ["proj", "pgd"])
def test_graphed_training_matches_eager(mode):
    """One CUDA graph per resident batch (first step eager + capture, then replays)
    follows the eager trainer's trajectory: same losses and parameters, step by step,
    over batches that alternate; a state load drops the captured steps."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.training import UnfoldedTrainer
    K, M, T, Bt = 8, 64, 10, 1024
    layer = capi.LAYER_PROJ if mode == "proj" else capi.LAYER_PGD
    a = 1.0 if mode == "proj" else 1 / 15
    t = torch.full((K,), 1.0 if mode == "proj" else math.sqrt(10.0), device="cuda")
    eager = UnfoldedTrainer(layer, T, K, M, Bt, a=a, lr=2e-3)
    graphed = UnfoldedTrainer(layer, T, K, M, Bt, a=a, lr=2e-3, graphs=True)
    batches = [eager.make_batch(i, seed=6) for i in range(3)]
    for i in range(9):
        le = eager.train_step(batches[i % 3], t)
        lg = graphed.train_step(batches[i % 3], t, sync=(i % 2 == 0))
        lg = float(lg)
        assert lg == pytest.approx(le, rel=1e-6, abs=0), (i, le, lg)
        assert torch.allclose(graphed.step, eager.step, rtol=1e-5, atol=0), i
        if mode == "pgd":
            assert torch.allclose(graphed.lam, eager.lam, rtol=1e-5, atol=0), i
    assert len(graphed._graphs) == 3
    state = graphed.state_dict()
    graphed.load_state_dict(state)
    assert len(graphed._graphs) == 0
    le = eager.train_step(batches[0], t)
    assert graphed.train_step(batches[0], t) == pytest.approx(le, rel=1e-6, abs=0)
    assert torch.allclose(graphed.step, eager.step, rtol=1e-5, atol=0)


def _train_step_one(plan, Hb, tb, step, lam, a, labels=None):
    """One instance (B = 1) through precode_train_step, or through
    precode_train_step_supervised with labels: (loss, dstep, dlam)."""
    from paper_2304_12745_gb300 import capi
    K, M = Hb.shape
    Hd = torch.from_numpy(Hb[None].astype(np.complex64)).cuda()
    td = torch.from_numpy(np.ascontiguousarray(tb, np.float32)).cuda()
    sd = torch.tensor(step, dtype=torch.float32, device="cuda")
    ld = torch.tensor(lam, dtype=torch.float32, device="cuda") if lam is not None else None
    loss = torch.empty(1, device="cuda")
    ds = torch.empty(len(step), device="cuda")
    dl = torch.empty(len(step), device="cuda") if lam is not None else None
    stream = torch.cuda.current_stream().cuda_stream
    if labels is None:
        capi.precode_train_step(plan.handle, M, K, 1, Hd, td, 0, sd, ld, a, loss, ds, dl, None, stream)
    else:
        Wd = torch.from_numpy(labels[None].astype(np.complex64)).cuda()
        capi.precode_train_step_supervised(plan.handle, M, K, 1, Hd, td, 0, Wd, sd, ld, loss, ds, dl,
                                           None, stream)
    torch.cuda.synchronize()
    return (float(loss.item()), ds.cpu().numpy().astype(np.float64),
            None if dl is None else dl.cpu().numpy().astype(np.float64))


PER_INSTANCE = [  # (layer, K, M, T, tensor cores, loss)
    ("proj", 8, 64, 10, True, "unsupervised"), ("proj", 8, 64, 10, True, "supervised"),
    # the split-FP16 kernel's checkpoints: 5 in tensor memory at T = 10 (every 2nd
    # layer) and T = 20 (every 4th), a global workspace at T = 40 (6 checkpoints)
    ("proj", 8, 64, 20, True, "unsupervised"), ("proj", 8, 64, 40, True, "unsupervised"),
    ("proj", 8, 64, 10, False, "supervised"), ("proj", 4, 32, 6, False, "unsupervised"),
    ("pgd", 8, 64, 20, True, "unsupervised"), ("pgd", 8, 64, 20, True, "supervised"),
    ("pgd", 4, 32, 20, False, "supervised")]


@pytest.mark.parametrize("layer,K,M,T,tc,kind", PER_INSTANCE)
def test_gradients_per_instance(orc, layer, K, M, T, tc, kind):
    """Loss and parameter gradients instance by instance (B = 1 calls), so that an
    error on a minority of instances cannot average out: the projected layer on
    8 dB log-normal user gains, the paper layer in the paper's setting (CN(0,1),
    gamma = 10 dB, I = 20 layers, eta in the clamp interval, lambda = 1/15).  The
    supervised cost (Sec. V) uses as labels the constrained optimum from the
    oracle's ADMM (O3), as the paper uses convex-solver solutions.  Per instance:
    the unsupervised loss within 1e-5 relative, the supervised one within what the
    W bar (1e-4) allows for a squared distance, each gradient within 2e-3 of the
    oracle's (relative to the instance's largest component)."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan
    rs = np.random.default_rng(60 + K + T)
    B0 = 24 if T <= 20 else 128  # longer runs pass near more shrink kinks: more candidates
    if layer == "proj":
        H = ch.lognormal(B0, K, M, seed=61 + K).astype(np.complex128)
        t = np.ones((B0, K))
        mu = ch.uniform_steps(T, 0.02, 0.08, seed=62).astype(np.float64)
        keep = _far_from_kinks_proj(orc, H, t, mu, 2e-5)
        mode, step, lam, a = capi.LAYER_PROJ, mu, None, 1.0
    else:
        H = ch.rayleigh(B0, K, M, seed=63 + K).astype(np.complex128)
        t = np.full((B0, K), math.sqrt(10.0))
        eta0 = ch.paper_eta(K, M)
        step = (eta0 * rs.uniform(0.5, 1.0, T)).astype(np.float32).astype(np.float64)
        lam = np.full(T, np.float32(1 / 15), np.float64)
        keep = _far_from_kinks_pgd(orc, H, t, step, lam, 2e-5)
        mode, a = capi.LAYER_PGD, 1 / 15
    idx = np.nonzero(keep)[0][:12]
    assert len(idx) >= 8
    plan = Plan(mode, T, [(M, K)], 1, tensor_cores=tc)
    if kind == "supervised":  # labels: the constrained optimum (ADMM), as the paper's CVXPY ones
        Wgt, _, st = orc.batch_admm(H[idx], t[idx], tol=1e-10, nthreads=8)
        assert np.all(st == orc.OK)
        Wgt = Wgt.astype(np.complex64)
    for n, b in enumerate(idx):
        labels = None
        if kind == "supervised":
            labels = Wgt[n]  # complex64, as the GPU sees them
            ref = (orc.ufproj_grad_supervised(H[b], t[b], step, labels) if layer == "proj"
                   else orc.ufpgd_grad_supervised(H[b], t[b], step, lam, labels))
            W_o = (orc.ufproj_forward(H[b], t[b], step)[0] if layer == "proj"
                   else orc.ufpgd_forward(H[b], t[b], step, lam))
            # |loss error| <= 2 ||W - W_gt|| ||dW|| + ||dW||^2 with ||dW|| <= 1e-4 ||W|| (the W bar)
            dw = 1e-4 * np.linalg.norm(W_o)
            ltol = 2 * math.sqrt(ref[0]) * dw + dw * dw
        else:
            ref = (orc.ufproj_grad(H[b], t[b], step, a) if layer == "proj"
                   else orc.ufpgd_grad(H[b], t[b], step, lam, a))
            ltol = 1e-5 * ref[0]
        loss, g, gl = _train_step_one(plan, H[b], t[b], step, lam, a, labels)
        assert abs(loss - ref[0]) <= ltol, (b, loss, ref[0], ltol)
        assert np.allclose(g, ref[1], rtol=2e-3, atol=2e-3 * np.abs(ref[1]).max()), (b, g, ref[1])
        if layer == "pgd":
            assert np.allclose(gl, ref[2], rtol=2e-3, atol=2e-3 * np.abs(ref[2]).max()), (b, gl, ref[2])
    plan.close()


def test_supervised_training_lowers_the_mse(orc):
    """Adam on the supervised cost (Sec. V) through the trainer: the projected
    layer's steps learned towards labels that are the layer's own output at other
    steps; the MSE falls to a fifth of its start (the steps themselves are not
    identifiable: several step vectors give nearly the same output)."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.training import UnfoldedTrainer
    K, M, T, B = 8, 64, 6, 256
    mu_true = np.linspace(0.09, 0.03, T).astype(np.float32)
    H = ch.rayleigh(B, K, M, seed=70)
    t = np.ones((B, K))
    Wl = orc.batch_forward(1, H.astype(np.complex128), t, mu_true.astype(np.float64), nthreads=8)[0]
    tr = UnfoldedTrainer(capi.LAYER_PROJ, T, K, M, B, a=1.0, lr=3e-3, init_step=[0.05] * T)
    Hd = torch.from_numpy(H).cuda()
    td = torch.ones(K, device="cuda")
    labels = torch.from_numpy(Wl.astype(np.complex64)).cuda()
    first = tr.train_step(Hd, td, labels=labels)
    for _ in range(150):
        last = tr.train_step(Hd, td, labels=labels)
    assert last < 0.2 * first, (first, last)
    assert np.all(tr.step.detach().cpu().numpy() >= 0)  # the projection mu >= 0 held
    tr.plan.close()


@pytest.mark.parametrize("K,M,tc", [(4, 32, False), (8, 64, True)])
def test_batch_means_at_long_depth_equal_per_instance_means(K, M, tc):
    """The batch loss and gradients are FP64 means of the per-instance values. At
    T = 130 the per-instance record holds 1 + 2T = 261 scalars, more than one
    reduction block has threads, and B = 300 leaves a ragged row chunk. The batch
    results must equal the mean of the same instances solved one at a time (B = 1,
    where the mean is the instance's own value), up to the final rounding to FP32.
    Uses the paper layer, so d lam is reduced as well."""
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan
    T, B = 130, 300
    H = ch.rayleigh(B, K, M, seed=90 + K)
    t = np.full((B, K), math.sqrt(10.0), np.float32)
    rs = np.random.default_rng(91)
    eta = (ch.paper_eta(K, M) * rs.uniform(0.5, 1.0, T)).astype(np.float32).astype(np.float64)
    lam = np.full(T, np.float32(1 / 15), np.float64)
    a = 1 / 15
    plan = Plan(capi.LAYER_PGD, T, [(M, K)], B, tensor_cores=tc)
    loss, ge, gl = _train_step(plan, H, t, eta, lam, a)
    one = [_train_step_one(plan, H[b], t[b], eta, lam, a) for b in range(B)]
    plan.close()
    per_loss = np.array([o[0] for o in one])
    per_ge = np.array([o[1] for o in one])
    per_gl = np.array([o[2] for o in one])
    assert np.all(np.isfinite(per_ge)) and np.all(np.isfinite(per_gl))
    assert loss == pytest.approx(per_loss.mean(), rel=1e-6)
    for got, per in ((ge, per_ge), (gl, per_gl)):
        assert np.allclose(got, per.mean(0), rtol=1e-6, atol=1e-9 * np.abs(per).max()), (got, per.mean(0))
