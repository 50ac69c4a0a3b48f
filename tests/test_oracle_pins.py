"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one oracle routine to something other than itself: a closed
form, an invariant, a library routine that computes the same object by a
different method (SVD pseudo-inverse, scipy minimisers), brute force on tiny
inputs, or a value the paper prints.  A plausible slip in the oracle (dropped
term, wrong sign, conjugate or transpose, wrong prox threshold, factor-2
convention) fails at least one of them.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest
from scipy import optimize

from paper_2304_12745_gb300 import channels as ch

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cn(rs, *shape):
    return (rs.standard_normal(shape) + 1j * rs.standard_normal(shape)) / np.sqrt(2)


def l21_np(W):
    return np.sqrt((np.abs(W) ** 2).sum(0)).sum()


def zf_pinv(H, t):
    """ZF from the SVD pseudo-inverse: W^T = H^+ S (minimum-norm solution of H W^T = S)."""
    return (np.linalg.pinv(H) @ np.diag(t)).T


# --------------------------------------------------------------------------- O5

def test_l21_and_residual_definitions(orc):
    rs = np.random.default_rng(0)
    H, W = cn(rs, 3, 5), cn(rs, 3, 5)
    t = np.array([1.0, 2.0, 0.5])
    assert orc.l21(W) == pytest.approx(l21_np(W), rel=1e-14)
    # column norms, not row norms: a matrix with one nonzero column has l21 = its norm
    C = np.zeros((3, 5), complex)
    C[:, 2] = [3, 4j, 0]
    assert orc.l21(C) == pytest.approx(5.0, rel=1e-15)
    R = H @ W.T - np.diag(t)
    assert orc.residual_fro(H, t, W) == pytest.approx(np.linalg.norm(R), rel=1e-13)
    assert np.allclose(orc.residual_matrix(H, t, W), R.T, atol=1e-13)


def test_gram_cholesky_and_singular(orc):
    rs = np.random.default_rng(1)
    H = cn(rs, 4, 9)
    G, L, st = orc.gram_cholesky(H)
    assert st == orc.OK
    assert np.allclose(G, H @ H.conj().T, atol=1e-13)
    assert np.allclose(L @ L.conj().T, G, atol=1e-12)
    assert np.allclose(np.triu(L, 1), 0) and np.all(np.diag(L).real > 0)
    Hs = H.copy()
    Hs[3] = Hs[1]  # two users with the same channel: rank K-1
    _, _, st = orc.gram_cholesky(Hs)
    assert st == orc.SINGULAR
    W, st = orc.ufproj_forward(Hs, np.ones(4), [0.1, 0.1])
    assert st == orc.SINGULAR and not np.any(W)


def test_zf_matches_svd_pseudoinverse(orc):
    rs = np.random.default_rng(2)
    for K, M in [(1, 5), (4, 32), (8, 64), (5, 5)]:
        H = cn(rs, K, M)
        t = rs.uniform(0.5, 2.0, K)
        W = orc.zf(H, t)
        assert np.allclose(W, zf_pinv(H, t), atol=1e-11)
        assert orc.residual_fro(H, t, W) < 1e-12


def test_prox_l21_is_the_proximal_map(orc):
    """prox_tau(v) = argmin_x tau*||x||_{2,1} + 0.5*||x - v||_F^2 per column (Sec. IV end)."""
    rs = np.random.default_rng(3)
    V = cn(rs, 2, 4) * np.array([0.1, 1.0, 2.0, 0.4])
    tau = 0.5
    P = orc.prox_l21(V, tau)
    for m in range(4):
        v = np.concatenate([V[:, m].real, V[:, m].imag])

        def f(x):
            return tau * np.linalg.norm(x) + 0.5 * np.sum((x - v) ** 2)

        best = optimize.minimize(f, v * 0.5, method="Nelder-Mead",
                                 options=dict(xatol=1e-12, fatol=1e-14, maxiter=20000))
        x = P[:, m]
        xr = np.concatenate([x.real, x.imag])
        assert f(xr) <= best.fun + 1e-10
        assert np.allclose(xr, best.x, atol=1e-5)
    # boundary ||v|| == tau gives 0; below gives 0; a column at 2*tau is halved
    e = np.zeros((2, 3), complex)
    e[0, 0], e[1, 1], e[0, 2] = tau, 0.3 * tau, 2 * tau
    P = orc.prox_l21(e, tau)
    assert P[0, 0] == 0 and P[1, 1] == 0 and P[0, 2] == pytest.approx(tau)


# --------------------------------------------------------------------------- O2 / p1, p4

def test_projection_idempotent_and_feasible(orc):
    """p4: P_A(P_A(X)) = P_A(X), H P_A(X)^T = S, and X - P_A(X) is orthogonal to A - P_A(X)."""
    rs = np.random.default_rng(4)
    H = cn(rs, 8, 64)
    t = np.full(8, math.sqrt(10))
    X = cn(rs, 8, 64)
    P1 = orc.project(H, t, X)
    P2 = orc.project(H, t, P1)
    assert np.linalg.norm(P2 - P1) / np.linalg.norm(P1) < 1e-12
    assert orc.residual_fro(H, t, P1) / np.linalg.norm(t) < 1e-12
    # orthogonality: for any feasible Y, Re<X - P1, Y - P1> = 0
    Y = orc.project(H, t, cn(rs, 8, 64))
    assert abs(np.vdot(X - P1, Y - P1).real) < 1e-10 * np.linalg.norm(X) * np.linalg.norm(Y)
    # same projection from the SVD pseudo-inverse: P_A(X) = X - (X H^T - S) (H^+)^T
    Pp = X - (X @ H.T - np.diag(t)) @ np.linalg.pinv(H).T
    assert np.allclose(P1, Pp, atol=1e-11)


def test_projected_layers_feasible_every_layer(orc):
    rs = np.random.default_rng(5)
    H = cn(rs, 4, 32)
    t = np.ones(4)
    mu = np.full(20, 0.05)
    W, st, tr = orc.ufproj_forward(H, t, mu, trace=True)
    assert st == orc.OK
    assert np.allclose(tr[0], zf_pinv(H, t), atol=1e-12)  # layer 0 is ZF
    for l in range(21):
        assert orc.residual_fro(H, t, tr[l]) < 1e-12
    # one layer = shrink then project, against the pseudo-inverse projector
    X = orc.prox_l21(tr[3], mu[3])
    Pp = X - (X @ H.T - np.diag(t)) @ np.linalg.pinv(H).T
    assert np.allclose(tr[4], Pp, atol=1e-11)
    # shrink makes progress on the objective from ZF at small mu
    assert orc.l21(tr[-1]) < orc.l21(tr[0])


def test_square_channel_leaves_no_freedom(orc):
    """p1: M = K, the feasible set is the single point W = (H^{-1} S)^T."""
    rs = np.random.default_rng(6)
    for K in (1, 3, 6):
        H = cn(rs, K, K)
        t = rs.uniform(0.5, 2.0, K)
        Wstar = np.linalg.solve(H, np.diag(t)).T
        W, st, tr = orc.ufproj_forward(H, t, np.full(7, 0.3), trace=True)
        for l in range(8):
            assert np.allclose(tr[l], Wstar, atol=1e-10)
        r = orc.admm_solve(H, t, rho=1.0, tol=1e-12)
        assert np.allclose(r["W"], Wstar, atol=1e-10)


# --------------------------------------------------------------------------- O3 / p2, p8, p9, p10

def test_single_user_constrained_closed_form(orc):
    """p2: K = 1 reduces to min ||w||_1 s.t. h^T w = s: all power on argmax |h_m|."""
    rs = np.random.default_rng(7)
    for M in (2, 5, 16):
        h = cn(rs, 1, M)
        s = np.array([1.7])
        mstar = int(np.argmax(np.abs(h[0])))
        r = orc.admm_solve(h, s, rho=1.0, tol=1e-13, max_iter=500000)
        W = r["W"]
        assert orc.l21(W) == pytest.approx(s[0] / np.abs(h[0]).max(), rel=1e-8)
        assert W[0, mstar] == pytest.approx(s[0] / h[0, mstar], rel=1e-7)
        assert np.abs(np.delete(W[0], mstar)).max() < 1e-7
        # projected layers with a diminishing shrink (sum mu = inf, sum mu^2 < inf)
        # approach the same optimum from the feasible side
        opt = s[0] / np.abs(h[0]).max()
        mu = 0.5 * opt / np.arange(1, 20001) ** 0.75
        Wl, _ = orc.ufproj_forward(h, s, mu)
        assert opt * (1 - 1e-12) <= orc.l21(Wl) <= opt * (1 + 2e-3)


def test_diminishing_projected_layers_approach_the_admm_optimum(orc):
    """Cross-check of the two constrained solvers at K > 1: projected layers with a
    diminishing shrink (sum mu = inf, sum mu^2 < inf) stay feasible and close in on
    the ADMM optimum from above as the number of layers grows."""
    rs = np.random.default_rng(20)
    for _ in range(3):
        K, M = 3, 12
        H = cn(rs, K, M)
        t = rs.uniform(0.5, 1.5, K)
        opt = orc.l21(orc.admm_solve(H, t, rho=1.0, tol=1e-13, max_iter=1000000)["W"])
        gaps = []
        for n in (2000, 100000):
            mu = 0.5 * opt / K / np.arange(1, n + 1) ** 0.75
            W, st = orc.ufproj_forward(H, t, mu)
            assert st == orc.OK and orc.residual_fro(H, t, W) < 1e-12
            gaps.append(orc.l21(W) / opt - 1)
        assert -1e-9 <= gaps[1] < gaps[0] and gaps[1] < 2e-4, gaps


def _nullspace(H):
    _, sv, Vh = np.linalg.svd(H)
    return Vh[H.shape[0]:].conj().T  # columns span {x : H x = 0}


@pytest.mark.parametrize("K,M,seed", [(1, 2, 8), (2, 3, 9), (1, 3, 10)])
def test_constrained_brute_force(orc, K, M, seed):
    """p8: grid + multi-start local refinement over the null-space parametrisation
    X = X0 + N C of {H X = S} (X = W^T), 2 (M-K) K real dimensions."""
    rs = np.random.default_rng(seed)
    H = cn(rs, K, M)
    t = rs.uniform(0.5, 1.5, K)
    X0 = zf_pinv(H, t).T  # M x K particular solution
    N = _nullspace(H)     # M x (M-K)
    d = N.shape[1]

    def obj(z):
        c = z[:d * K] + 1j * z[d * K:]
        X = X0 + N @ c.reshape(d, K)
        return np.sqrt((np.abs(X) ** 2).sum(1)).sum()

    nz = 2 * d * K
    span = 2.0 * np.abs(X0).max()
    grid = np.linspace(-span, span, 15 if nz <= 2 else 9)
    pts = sorted((obj(np.array(z)), z) for z in itertools.product(grid, repeat=nz))[:8]
    best = np.inf
    for _, z0 in pts:
        res = optimize.minimize(obj, np.array(z0), method="Nelder-Mead",
                                options=dict(xatol=1e-13, fatol=1e-15, maxiter=200000,
                                             maxfev=200000))
        for _ in range(3):
            res = optimize.minimize(obj, res.x, method="Nelder-Mead",
                                    options=dict(xatol=1e-13, fatol=1e-15, maxiter=200000,
                                                 maxfev=200000))
        best = min(best, res.fun)
    r = orc.admm_solve(H, t, rho=1.0, tol=1e-13, max_iter=1000000)
    assert orc.residual_fro(H, t, r["W"]) < 1e-12
    assert orc.l21(r["W"]) <= best * (1 + 1e-9)
    assert orc.l21(r["W"]) == pytest.approx(best, rel=1e-6)


def test_admm_kkt_certificate(orc):
    """p9: exists Lambda with -(Lambda H^*)_m = w_m/||w_m|| on the support, ||(Lambda H^*)_m|| <= 1 off it."""
    rs = np.random.default_rng(11)
    H = cn(rs, 4, 24)
    t = np.full(4, math.sqrt(10))
    r = orc.admm_solve(H, t, rho=1.0, tol=1e-13, max_iter=1000000)
    Z = r["Z"]
    cn_ = np.sqrt((np.abs(Z) ** 2).sum(0))
    supp = cn_ > 1e-9 * cn_.max()
    assert 4 <= supp.sum() < 24  # sparse, and at least K antennas on
    target = -(Z[:, supp] / cn_[supp])            # K x |supp|
    A = H.conj()[:, supp]                          # Lambda @ A = target
    Lam, *_ = np.linalg.lstsq(A.T, target.T, rcond=None)
    Lam = Lam.T
    stat = np.linalg.norm(Lam @ A - target) / np.sqrt(supp.sum())
    assert stat < 1e-6
    off = np.linalg.norm((Lam @ H.conj())[:, ~supp], axis=0)
    assert np.all(off <= 1 + 1e-6)
    # the ADMM dual agrees: rho*U is the same subgradient
    G = r["rho"] * r["U"]
    assert np.allclose(G[:, supp], (Z[:, supp] / cn_[supp]), atol=1e-5)


def test_constrained_optimum_reproduces_paper_pcg(orc):
    """p10: mean PCG of the exact optimum over i.i.d. CN(0,1) channels, K=8, M=64,
    gamma = 10 dB, sigma_nu = 1, against the paper's convex-solver value."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["pcg_constrained_optimum"]
    B, K, M = 400, gold["K"], gold["M"]
    H = ch.rayleigh(B, K, M, seed=1234).astype(np.complex128)
    t = ch.targets(B, K, gamma_db=gold["gamma_db"], sigma_nu=gold["sigma_nu"]).astype(np.float64)
    W, iters, st = orc.batch_admm(H, t, rho=1.0, tol=1e-10, nthreads=os.cpu_count() or 1)
    assert np.all(st == 0)
    p = np.array([orc.pcg(H[b], t[b], W[b]) for b in range(B)])
    se = p.std() / np.sqrt(B)
    # the paper averages 5000 channels (s.e. ~ 4e-4); allow 4 of our s.e. plus that
    assert abs(p.mean() - gold["value"]) < 4 * se + 0.0015, (p.mean(), se)
    assert np.all(p >= 1.0 - 1e-9)  # never worse than ZF: ZF is feasible


# --------------------------------------------------------------------------- O1 / O4 / p3, p5, p6, p7

def test_single_user_penalised_closed_form_and_factor_two(orc):
    """p3: K = 1, the paper's iteration converges to the minimiser of
    2*lam*||w||_1 + |h^T w - s|^2: w_{m*} = c / h_{m*}, c = (1 - lam/(a|s|))_+ s."""
    rs = np.random.default_rng(12)
    h = cn(rs, 1, 6)
    s = np.array([2.0])
    lam = 0.3
    a = np.abs(h[0]).max()
    mstar = int(np.argmax(np.abs(h[0])))
    eta = 1.0 / orc.lambda_max(h)
    W, it = orc.pgd_longrun(h, s, eta, lam, tol=1e-15, max_iter=5_000_000)
    c = max(0.0, 1 - lam / (a * s[0])) * s[0]
    assert W[0, mstar] == pytest.approx(c / h[0, mstar], rel=1e-8)
    assert np.abs(np.delete(W[0], mstar)).max() < 1e-9
    # the convention without the factor 2 would give a different point
    c_alt = max(0.0, 1 - lam / (2 * a * s[0])) * s[0]
    assert abs(abs(W[0, mstar]) - abs(c_alt / h[0, mstar])) > 1e-3


def test_penalised_brute_force(orc):
    """p8 (penalised): K=1, M=2, 4 real dimensions, against the long-run PGD."""
    rs = np.random.default_rng(13)
    h = cn(rs, 1, 2)
    s = np.array([1.0])
    lam = 0.2

    def F(z):
        w = z[:2] + 1j * z[2:]
        return 2 * lam * np.abs(w).sum() + abs(h[0] @ w - s[0]) ** 2

    g = np.linspace(-2, 2, 13)
    best = min((F(np.array(z)), z) for z in itertools.product(g, repeat=4))
    res = optimize.minimize(F, np.array(best[1]), method="Nelder-Mead",
                            options=dict(xatol=1e-12, fatol=1e-15, maxiter=100000))
    W, _ = orc.pgd_longrun(h, s, 1.0 / orc.lambda_max(h), lam, tol=1e-15)
    val = orc.penalised_objective(h, s, lam, W)
    assert val == pytest.approx(F(np.concatenate([W[0].real, W[0].imag])), rel=1e-12)
    assert val <= res.fun + 1e-10
    assert val == pytest.approx(res.fun, rel=1e-7)


def test_paper_layer_monotone_descent(orc):
    """p5: with fixed eta <= 1/lambda_max(G), F_P = 2 lam ||W||_{2,1} + ||H W^T - S||^2 never increases."""
    rs = np.random.default_rng(14)
    H = cn(rs, 8, 64)
    t = np.full(8, math.sqrt(10))
    lam = 1 / 15
    eta = 1.0 / orc.lambda_max(H)
    T = 60
    _, tr = orc.ufpgd_forward(H, t, np.full(T, eta), np.full(T, lam), trace=True)
    F = [orc.penalised_objective(H, t, lam, tr[i]) for i in range(T + 1)]
    assert all(F[i + 1] <= F[i] + 1e-12 for i in range(T))
    assert F[-1] < 0.5 * F[0]
    # lambda_max itself against numpy
    assert orc.lambda_max(H) == pytest.approx(np.linalg.eigvalsh(H @ H.conj().T).max(), rel=1e-12)


def test_paper_layer_one_step_and_lambda_zero_limit(orc):
    """p7: lam = 0: one layer is H^* - eta (H^* H^T H^* - S H^*); many layers -> ZF."""
    rs = np.random.default_rng(15)
    H = cn(rs, 4, 32)
    t = np.array([1.0, 0.5, 2.0, 1.5])
    eta = ch.paper_eta(4, 32)
    W1 = orc.ufpgd_forward(H, t, [eta], [0.0])
    Hc = H.conj()
    assert np.allclose(W1, Hc - eta * (Hc @ H.T @ Hc - np.diag(t) @ Hc), atol=1e-12)
    # one layer with lam > 0 applies the column prox with threshold lam*eta
    lam = 2.0
    W1p = orc.ufpgd_forward(H, t, [eta], [lam])
    V = Hc - eta * (Hc @ H.T @ Hc - np.diag(t) @ Hc)
    r = np.linalg.norm(V, axis=0)
    f = np.where(r > lam * eta, 1 - lam * eta / r, 0.0)
    assert np.allclose(W1p, V * f, atol=1e-12)
    Wn = orc.ufpgd_forward(H, t, np.full(4000, 1.0 / orc.lambda_max(H)), np.zeros(4000))
    assert np.allclose(Wn, zf_pinv(H, t), atol=1e-9)


def test_feasible_precoder_hits_paper_sum_rate(orc):
    """p6: any feasible W gives SINR_k = gamma_k, so R_sum = sum log2(1 + gamma_k);
    for K = 8 and 10 dB the paper prints 27.68 bits/symbol."""
    gold = json.load(open(os.path.join(GOLDEN, "paper_values.json")))["target_sum_rate"]
    K = gold["K"]
    H = ch.rayleigh(3, K, 64, seed=77).astype(np.complex128)
    gamma = 10 ** (gold["gamma_db"] / 10)
    t = np.full((3, K), math.sqrt(gamma))  # t_k = sigma_nu sqrt(gamma_k), sigma_nu = 1, in FP64
    exact = K * math.log2(1 + gamma)
    assert round(exact, gold["digits"]) == gold["value"]
    for b in range(3):
        for W in (orc.zf(H[b], t[b]), orc.ufproj_forward(H[b], t[b], np.full(10, 0.2))[0],
                  orc.admm_solve(H[b], t[b], tol=1e-11)["W"]):
            assert orc.sum_rate(H[b], W, 1.0) == pytest.approx(exact, abs=1e-9)
            assert np.allclose(orc.sinr(H[b], W, 1.0), 10.0, rtol=1e-9)
    # an infeasible precoder (the paper layer after one step) does not land on it
    W = orc.ufpgd_forward(H[0], t[0], [ch.paper_eta(K, 64)], [1 / 15])
    assert abs(orc.sum_rate(H[0], W, 1.0) - exact) > 0.1
    # the targets scale with the noise amplitude, t_k = sigma_nu sqrt(gamma_k), so a
    # feasible precoder meets gamma_k at any sigma_nu (here 0.5 and 3)
    for sig in (0.5, 3.0):
        ts = sig * t[1]
        W = orc.zf(H[1], ts)
        assert np.allclose(orc.sinr(H[1], W, sig), gamma, rtol=1e-9)
        assert orc.sum_rate(H[1], W, sig) == pytest.approx(exact, abs=1e-9)


def test_pcg_definition(orc):
    rs = np.random.default_rng(16)
    H = cn(rs, 3, 12)
    t = np.ones(3)
    Wz = zf_pinv(H, t)
    assert orc.pcg(H, t, Wz) == pytest.approx(1.0, rel=1e-12)
    assert orc.pcg(H, t, 2 * Wz) == pytest.approx(0.5, rel=1e-12)


# --------------------------------------------------------------------------- O6 / p11

def _fd(f, x, h=1e-3):
    g = np.zeros_like(x)
    for i in range(len(x)):
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        g[i] = (f(xp) - f(xm)) / (2 * h)
    return g


def _min_kink_distance_proj(orc, H, t, mu):
    _, _, tr = orc.ufproj_forward(H, t, mu, trace=True)
    return min(np.abs(np.linalg.norm(tr[l], axis=0) - mu[l]).min() for l in range(len(mu)))


def test_projected_layer_gradient_vs_central_differences(orc):
    rs = np.random.default_rng(17)
    tested = 0
    for trial in range(40):
        H = cn(rs, 4, 12)
        t = np.ones(4)
        mu = rs.uniform(0.01, 0.1, 4)
        a = 1.0
        if _min_kink_distance_proj(orc, H, t, mu) < 4e-3:
            continue  # a column within reach of the kink r = mu: reported, not gated
        loss, g = orc.ufproj_grad(H, t, mu, a)
        gfd = _fd(lambda m: orc.ufproj_grad(H, t, m, a)[0], mu)
        assert np.allclose(g, gfd, rtol=1e-5, atol=1e-7 * abs(loss)), (g, gfd)
        tested += 1
    assert tested >= 3


def test_paper_layer_gradient_vs_central_differences(orc):
    rs = np.random.default_rng(18)
    K, M, T = 4, 16, 5
    eta0 = ch.paper_eta(K, M)
    tested = 0
    for trial in range(12):
        H = cn(rs, K, M)
        t = np.ones(K)
        eta = eta0 * rs.uniform(0.5, 1.0, T)
        lam = rs.uniform(0.5, 3.0, T)
        a = 1 / 15
        _, tr = orc.ufpgd_forward(H, t, eta, lam, trace=True)
        # distance of every pre-shrink column norm to its threshold
        dmin = np.inf
        for l in range(T):
            V = tr[l] - eta[l] * ((tr[l] @ H.T - np.diag(t)) @ H.conj())
            dmin = min(dmin, np.abs(np.linalg.norm(V, axis=0) - lam[l] * eta[l]).min())
        if dmin < 5e-3:
            continue
        loss, de, dl = orc.ufpgd_grad(H, t, eta, lam, a)
        fe = _fd(lambda e: orc.ufpgd_grad(H, t, e, lam, a)[0], eta, h=1e-6)
        fl = _fd(lambda x: orc.ufpgd_grad(H, t, eta, x, a)[0], lam, h=1e-3)
        assert np.allclose(de, fe, rtol=1e-5, atol=1e-8 * abs(loss) / eta0), (de, fe)
        assert np.allclose(dl, fl, rtol=1e-5, atol=1e-9 * abs(loss)), (dl, fl)
        tested += 1
    assert tested >= 3


def test_supervised_loss_gradients(orc):
    """Supervised cost of Sec. V, ||W_T - W_gt||_F^2: its value is the squared
    distance of the forward output to the label (definition); at parameters whose
    own output is the label the loss and every gradient vanish (a minimum); and
    the reverse mode agrees with central differences through both layer maps."""
    rs = np.random.default_rng(23)
    K, M, T = 4, 12, 4
    # projected layer
    tested = 0
    for trial in range(30):
        H = cn(rs, K, M)
        t = np.ones(K)
        mu = rs.uniform(0.01, 0.1, T)
        if _min_kink_distance_proj(orc, H, t, mu) < 4e-3:
            continue
        Wref = orc.ufproj_forward(H, t, rs.uniform(0.01, 0.1, T))[0]
        loss, g = orc.ufproj_grad_supervised(H, t, mu, Wref)
        W = orc.ufproj_forward(H, t, mu)[0]
        assert abs(loss - np.linalg.norm(W - Wref) ** 2) <= 1e-12 * max(loss, 1.0)
        gfd = _fd(lambda m: orc.ufproj_grad_supervised(H, t, m, Wref)[0], mu, h=1e-6)
        assert np.allclose(g, gfd, rtol=1e-5, atol=1e-7 * abs(loss)), (g, gfd)
        l0, g0 = orc.ufproj_grad_supervised(H, t, mu, W)
        assert l0 == 0.0 and np.all(g0 == 0.0)
        tested += 1
    assert tested >= 3
    # paper layer
    eta0 = ch.paper_eta(K, M)
    tested = 0
    for trial in range(12):
        H = cn(rs, K, M)
        t = np.ones(K)
        eta = eta0 * rs.uniform(0.5, 1.0, T)
        lam = rs.uniform(0.5, 3.0, T)
        _, tr = orc.ufpgd_forward(H, t, eta, lam, trace=True)
        dmin = np.inf
        for l in range(T):
            V = tr[l] - eta[l] * ((tr[l] @ H.T - np.diag(t)) @ H.conj())
            dmin = min(dmin, np.abs(np.linalg.norm(V, axis=0) - lam[l] * eta[l]).min())
        if dmin < 5e-3:
            continue
        Wref = orc.ufpgd_forward(H, t, eta0 * rs.uniform(0.5, 1.0, T), rs.uniform(0.5, 3.0, T))
        loss, de, dl = orc.ufpgd_grad_supervised(H, t, eta, lam, Wref)
        assert abs(loss - np.linalg.norm(tr[T] - Wref) ** 2) <= 1e-12 * max(loss, 1.0)
        fe = _fd(lambda e: orc.ufpgd_grad_supervised(H, t, e, lam, Wref)[0], eta, h=1e-6)
        fl = _fd(lambda x: orc.ufpgd_grad_supervised(H, t, eta, x, Wref)[0], lam, h=1e-3)
        assert np.allclose(de, fe, rtol=1e-5, atol=1e-8 * abs(loss) / eta0), (de, fe)
        assert np.allclose(dl, fl, rtol=1e-5, atol=1e-9 * abs(loss)), (dl, fl)
        l0, d0e, d0l = orc.ufpgd_grad_supervised(H, t, eta, lam, tr[T])
        assert l0 == 0.0 and np.all(d0e == 0.0) and np.all(d0l == 0.0)
        tested += 1
    assert tested >= 3


# --------------------------------------------------------------------------- batch harness

def test_batch_forward_matches_single_instances(orc):
    """The threaded batch harness runs the unchanged per-instance routines: its W, objective
    and residual equal single-instance calls for both layers, whatever the thread count."""
    rs = np.random.default_rng(19)
    B, K, M, T = 7, 3, 10, 4
    H = cn(rs, B, K, M)
    t = rs.uniform(0.5, 2.0, (B, K))
    eta = np.full(T, ch.paper_eta(K, M))
    lam = rs.uniform(0.1, 1.0, T)
    mu = rs.uniform(0.01, 0.1, T)
    for mode, p1, p2 in ((0, eta, lam), (1, mu, None)):
        for nthreads in (1, 3):
            W, obj, res, st = orc.batch_forward(mode, H, t, p1, p2, nthreads=nthreads)
            assert np.all(st == orc.OK)
            for b in range(B):
                Wb = (orc.ufpgd_forward(H[b], t[b], eta, lam) if mode == 0
                      else orc.ufproj_forward(H[b], t[b], mu)[0])
                assert np.array_equal(W[b], Wb)
                assert obj[b] == orc.l21(Wb)
                assert res[b] == orc.residual_fro(H[b], t[b], Wb)
