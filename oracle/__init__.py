"""FP64 CPU oracle for the deep-unfolded PA-consumption precoder (arXiv 2304.12745).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py``.  The GPU library never imports this package, and
this package shares no code with it.  The arithmetic lives in ``oracle.cpp``
(plain single-threaded FP64 C++); this module only marshals numpy arrays through
ctypes.

Functions and the passages they follow:
  ufpgd_forward   Sec. V, Eq. (unfoldednet), gradient of Sec. IV, l2,1 prox (Sec. IV)
  ufproj_forward  projected layer: group shrink + projection onto {H W^T = S}, Eq. (optim1)
  admm_solve      long-run solve of Eq. (optim1)
  pgd_longrun     long-run PGD, Eq. (proxgd), constant eta / lambda
  l21, residual_fro, sinr, sum_rate, zf, pcg   Eq. (effmodel), Sec. VI-B
  ufproj_grad, ufpgd_grad   reverse mode of the unsupervised loss of Sec. V
  ufproj_grad_supervised, ufpgd_grad_supervised   the same for the supervised loss
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")

OK = 0
SINGULAR = 2


def build(force: bool = False) -> str:
    """Compile ``oracle.cpp`` into ``liboracle.so`` (g++, -O2, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread",
             _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _declare(_lib)
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_L = ctypes.POINTER(ctypes.c_long)
_i, _l, _d = ctypes.c_int, ctypes.c_long, ctypes.c_double


def _declare(L):
    sig = {
        "orc_l21": (_d, [_i, _i, _D]),
        "orc_residual_fro": (_d, [_i, _i, _D, _D, _D]),
        "orc_residual_matrix": (None, [_i, _i, _D, _D, _D, _D]),
        "orc_sinr": (None, [_i, _i, _D, _D, _d, _D]),
        "orc_sum_rate": (_d, [_i, _i, _D, _D, _d]),
        "orc_gram_cholesky": (_i, [_i, _i, _D, _D, _D]),
        "orc_zf": (_i, [_i, _i, _D, _D, _D]),
        "orc_pcg": (_d, [_i, _i, _D, _D, _D]),
        "orc_project": (_i, [_i, _i, _D, _D, _D]),
        "orc_prox_l21": (None, [_i, _i, _D, _d]),
        "orc_ufpgd_forward": (_i, [_i, _i, _D, _D, _i, _D, _D, _D, _D, _D]),
        "orc_ufproj_forward": (_i, [_i, _i, _D, _D, _i, _D, _D, _D]),
        "orc_admm_solve": (_i, [_i, _i, _D, _D, _D, _l, _d, _D, _D, _D, _L]),
        "orc_lambda_max": (_d, [_i, _i, _D]),
        "orc_pgd_longrun": (_i, [_i, _i, _D, _D, _d, _d, _l, _d, _D, _D, _L]),
        "orc_penalised_objective": (_d, [_i, _i, _D, _D, _d, _D]),
        "orc_ufproj_grad": (_i, [_i, _i, _D, _D, _i, _D, _d, _D, _D]),
        "orc_ufpgd_grad": (_i, [_i, _i, _D, _D, _i, _D, _D, _d, _D, _D, _D]),
        "orc_ufproj_grad_loss": (_i, [_i, _i, _D, _D, _i, _D, _d, _D, _D, _D]),
        "orc_ufpgd_grad_loss": (_i, [_i, _i, _D, _D, _i, _D, _D, _d, _D, _D, _D, _D]),
        "orc_batch_forward": (_i, [_i, _i, _l, _i, _i, _D, _D, _i, _D, _D, _D, _D, _D, _I]),
        "orc_batch_admm": (_i, [_i, _l, _i, _i, _D, _D, _d, _l, _d, _D, _L, _I]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _r(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _shape(H):
    H = _c(H)
    assert H.ndim == 2
    return H, H.shape[0], H.shape[1]


# ------------------------------------------------------------------ metrics (O5)

def l21(W) -> float:
    W, K, M = _shape(W)
    return lib().orc_l21(K, M, _p(W))


def residual_fro(H, t, W) -> float:
    H, K, M = _shape(H)
    return lib().orc_residual_fro(K, M, _p(H), _p(_r(t)), _p(_c(W)))


def residual_matrix(H, t, W) -> np.ndarray:
    H, K, M = _shape(H)
    E = np.zeros((K, K), np.complex128)
    lib().orc_residual_matrix(K, M, _p(H), _p(_r(t)), _p(_c(W)), _p(E))
    return E


def sinr(H, W, sigma: float = 1.0) -> np.ndarray:
    H, K, M = _shape(H)
    out = np.zeros(K)
    lib().orc_sinr(K, M, _p(H), _p(_c(W)), sigma, _p(out))
    return out


def sum_rate(H, W, sigma: float = 1.0) -> float:
    H, K, M = _shape(H)
    return lib().orc_sum_rate(K, M, _p(H), _p(_c(W)), sigma)


def gram_cholesky(H):
    H, K, M = _shape(H)
    G = np.zeros((K, K), np.complex128)
    Lf = np.zeros((K, K), np.complex128)
    st = lib().orc_gram_cholesky(K, M, _p(H), _p(G), _p(Lf))
    return G, Lf, st


def zf(H, t) -> np.ndarray:
    H, K, M = _shape(H)
    W = np.zeros((K, M), np.complex128)
    st = lib().orc_zf(K, M, _p(H), _p(_r(t)), _p(W))
    if st != OK:
        raise np.linalg.LinAlgError("Gram matrix singular")
    return W


def pcg(H, t, W) -> float:
    H, K, M = _shape(H)
    return lib().orc_pcg(K, M, _p(H), _p(_r(t)), _p(_c(W)))


def project(H, t, X) -> np.ndarray:
    H, K, M = _shape(H)
    X = _c(X).copy()
    st = lib().orc_project(K, M, _p(H), _p(_r(t)), _p(X))
    if st != OK:
        raise np.linalg.LinAlgError("Gram matrix singular")
    return X


def prox_l21(W, tau: float) -> np.ndarray:
    W, K, M = _shape(W)
    W = W.copy()
    lib().orc_prox_l21(K, M, _p(W), tau)
    return W


# ------------------------------------------------------------------ O1 / O2

def ufpgd_forward(H, t, eta, lam, W0=None, trace: bool = False):
    """Paper layer (Eq. unfoldednet), T = len(eta) layers; W0 None -> H^*."""
    H, K, M = _shape(H)
    eta, lam = _r(eta), _r(lam)
    T = len(eta)
    assert len(lam) == T
    W = np.zeros((K, M), np.complex128)
    tr = np.zeros((T + 1, K, M), np.complex128) if trace else None
    w0 = _c(W0) if W0 is not None else None
    lib().orc_ufpgd_forward(K, M, _p(H), _p(_r(t)), T, _p(eta), _p(lam), _p(w0), _p(W), _p(tr))
    return (W, tr) if trace else W


def ufproj_forward(H, t, mu, trace: bool = False):
    """Projected layer, T = len(mu) layers from the ZF point.  Returns (W, status[, trace])."""
    H, K, M = _shape(H)
    mu = _r(mu)
    T = len(mu)
    W = np.zeros((K, M), np.complex128)
    tr = np.zeros((T + 1, K, M), np.complex128) if trace else None
    st = lib().orc_ufproj_forward(K, M, _p(H), _p(_r(t)), T, _p(mu), _p(W), _p(tr))
    return (W, st, tr) if trace else (W, st)


# ------------------------------------------------------------------ O3 / O4

def admm_solve(H, t, rho: float = 1.0, max_iter: int = 200000, tol: float = 1e-12):
    """Returns dict(W, Z, U, rho, iters, status)."""
    H, K, M = _shape(H)
    W = np.zeros((K, M), np.complex128)
    Z = np.zeros_like(W)
    U = np.zeros_like(W)
    r = ctypes.c_double(rho)
    it = ctypes.c_long(0)
    st = lib().orc_admm_solve(K, M, _p(H), _p(_r(t)), ctypes.byref(r), max_iter, tol, _p(W),
                              _p(Z), _p(U), ctypes.byref(it))
    return dict(W=W, Z=Z, U=U, rho=r.value, iters=it.value, status=st)


def lambda_max(H) -> float:
    H, K, M = _shape(H)
    return lib().orc_lambda_max(K, M, _p(H))


def pgd_longrun(H, t, eta: float, lam: float, max_iter: int = 10_000_000, tol: float = 1e-14,
                W0=None):
    H, K, M = _shape(H)
    W = np.zeros((K, M), np.complex128)
    it = ctypes.c_long(0)
    w0 = _c(W0) if W0 is not None else None
    lib().orc_pgd_longrun(K, M, _p(H), _p(_r(t)), eta, lam, max_iter, tol, _p(w0), _p(W),
                          ctypes.byref(it))
    return W, it.value


def penalised_objective(H, t, lam: float, W) -> float:
    H, K, M = _shape(H)
    return lib().orc_penalised_objective(K, M, _p(H), _p(_r(t)), lam, _p(_c(W)))


# ------------------------------------------------------------------ O6

def ufproj_grad(H, t, mu, a: float):
    """(loss, dloss/dmu) for loss = a*||W_T||_{2,1} + ||H W_T^T - S||_F^2."""
    H, K, M = _shape(H)
    mu = _r(mu)
    T = len(mu)
    loss = ctypes.c_double(0.0)
    dmu = np.zeros(T)
    st = lib().orc_ufproj_grad(K, M, _p(H), _p(_r(t)), T, _p(mu), a, ctypes.byref(loss), _p(dmu))
    if st != OK:
        raise np.linalg.LinAlgError("Gram matrix singular")
    return loss.value, dmu


def ufpgd_grad(H, t, eta, lam, a: float):
    """(loss, dloss/deta, dloss/dlam) through the paper layers from W^(0) = H^*."""
    H, K, M = _shape(H)
    eta, lam = _r(eta), _r(lam)
    T = len(eta)
    loss = ctypes.c_double(0.0)
    de, dl = np.zeros(T), np.zeros(T)
    lib().orc_ufpgd_grad(K, M, _p(H), _p(_r(t)), T, _p(eta), _p(lam), a, ctypes.byref(loss),
                         _p(de), _p(dl))
    return loss.value, de, dl


def ufproj_grad_supervised(H, t, mu, Wgt):
    """(loss, dloss/dmu) for the supervised loss ||W_T - W_gt||_F^2 (Sec. V)."""
    H, K, M = _shape(H)
    mu = _r(mu)
    T = len(mu)
    Wgt = _c(Wgt)
    assert Wgt.shape == (K, M)
    loss = ctypes.c_double(0.0)
    dmu = np.zeros(T)
    st = lib().orc_ufproj_grad_loss(K, M, _p(H), _p(_r(t)), T, _p(mu), 0.0, _p(Wgt),
                                    ctypes.byref(loss), _p(dmu))
    if st != OK:
        raise np.linalg.LinAlgError("Gram matrix singular")
    return loss.value, dmu


def ufpgd_grad_supervised(H, t, eta, lam, Wgt):
    """(loss, dloss/deta, dloss/dlam) for ||W_T - W_gt||_F^2 through the paper layers."""
    H, K, M = _shape(H)
    eta, lam = _r(eta), _r(lam)
    T = len(eta)
    Wgt = _c(Wgt)
    assert Wgt.shape == (K, M)
    loss = ctypes.c_double(0.0)
    de, dl = np.zeros(T), np.zeros(T)
    lib().orc_ufpgd_grad_loss(K, M, _p(H), _p(_r(t)), T, _p(eta), _p(lam), 0.0, _p(Wgt),
                              ctypes.byref(loss), _p(de), _p(dl))
    return loss.value, de, dl


# ------------------------------------------------------------------ batch harness

def batch_forward(mode: int, H, t, p1, p2=None, nthreads: int = 1):
    """Run O1 (mode 0) or O2 (mode 1) on H: [B][K][M].  Returns W, obj, resid, status."""
    H = _c(H)
    B, K, M = H.shape
    t = _r(t)
    assert t.shape == (B, K)
    p1 = _r(p1)
    T = len(p1)
    p2 = _r(p2) if p2 is not None else np.zeros(T)
    W = np.zeros_like(H)
    obj = np.zeros(B)
    res = np.zeros(B)
    st = np.zeros(B, np.int32)
    lib().orc_batch_forward(mode, nthreads, B, K, M, _p(H), _p(t), T, _p(p1), _p(p2), _p(W),
                            _p(obj), _p(res), st.ctypes.data_as(_I))
    return W, obj, res, st


def batch_admm(H, t, rho: float = 1.0, max_iter: int = 200000, tol: float = 1e-10,
               nthreads: int = 1):
    H = _c(H)
    B, K, M = H.shape
    t = _r(t)
    W = np.zeros_like(H)
    iters = np.zeros(B, np.int64)
    st = np.zeros(B, np.int32)
    lib().orc_batch_admm(nthreads, B, K, M, _p(H), _p(t), rho, max_iter, tol, _p(W),
                         iters.ctypes.data_as(_L), st.ctypes.data_as(_I))
    return W, iters, st
