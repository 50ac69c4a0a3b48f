// FP64 CPU oracle for the deep-unfolded PA-consumption precoder
// (Feys, Mestre, Peschiera, Rottenberg, "Deep Unfolding for Fast Linear Massive
// MIMO Precoders under a PA Consumption Model", VTC2023-Spring, arXiv 2304.12745).
//
// TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
// CUDA path is checked against.  Only the test-suite, the smoke check and the
// benchmark's CPU-baseline leg load it.  It shares no code, header, table or
// helper with the GPU library, and the GPU library never calls it.
//
// Everything is plain single-threaded IEEE FP64 (std::complex<double>), compiled
// with -ffp-contract=off, loops written in the order the paper states the maths.
// The only parallelism is `orc_batch_*`, which runs the unchanged per-instance
// routine on disjoint instance ranges, one std::thread each.
//
// Notation (paper Sec. II-III): K users, M antennas, H in C^{K x M} (row k is
// user k), W in C^{K x M} (column m is antenna m), x = W^T s, S = sigma_nu
// D_gamma^{1/2} is a real K x K diagonal passed as its diagonal t[k] > 0.
// Storage: row-major [K][M] complex, interleaved (re, im) doubles.
//
// Contents
//   O1  orc_ufpgd_forward     paper layer, Eq. (unfoldednet) with Eq. (proxgd)'s
//                             gradient (Sec. IV) and the l2,1 prox (Sec. IV end).
//   O2  orc_ufproj_forward    projected layer: group shrink, then orthogonal
//                             projection onto {W : H W^T = S} through the Gram
//                             Cholesky factor (problem Eq. (optim1)).
//   O3  orc_admm_solve        long-run solve of Eq. (optim1) (ADMM on W = Z).
//   O4  orc_pgd_longrun       long-run PGD of Eq. (proxgd) with fixed eta, lambda.
//   O5  metrics               ||W||_{2,1} (Eq. effmodel), residual, SINR, R_sum,
//                             ZF precoder and PCG (Sec. VI-B).
//   O6  gradients             reverse mode of the unsupervised and the supervised
//                             loss (Sec. V) through both layer maps.
//
// Readings of the paper taken here (each also listed in the design notes):
//   * the gradient of f(W) = ||H W^T - S||_F^2 is the Wirtinger derivative
//     (W H^T - S) H^* used literally (Sec. IV), so a fixed point of the paper's
//     iteration minimises 2*lambda*||W||_{2,1} + f(W);
//   * sigma_nu enters S as an amplitude; the caller passes t_k = sigma_nu sqrt(gamma_k);
//   * prox at ||v_m|| == tau returns 0 (both branches of the prox agree there);
//   * the projected layer shrinks first and projects second, so every output
//     satisfies H W^T = S; its initial point is the ZF precoder S G^{-T} H^*.

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

using cd = std::complex<double>;

constexpr int ORC_OK = 0;
constexpr int ORC_SINGULAR = 2;
constexpr int ORC_EINVAL = 22;

inline const cd* as_c(const double* p) { return reinterpret_cast<const cd*>(p); }
inline cd* as_c(double* p) { return reinterpret_cast<cd*>(p); }

// ---------------------------------------------------------------- O5 pieces

// ||W||_{2,1} = sum_m sqrt(sum_k |w_{k,m}|^2)   (Eq. effmodel, alpha = 1)
double l21(int K, int M, const cd* W) {
  double s = 0.0;
  for (int m = 0; m < M; ++m) {
    double p = 0.0;
    for (int k = 0; k < K; ++k) p += std::norm(W[k * M + m]);
    s += std::sqrt(p);
  }
  return s;
}

// E = W H^T - S   (K x K).  This is (H W^T - S)^T because S is diagonal.
void residual_matrix(int K, int M, const cd* W, const cd* H, const double* t, cd* E) {
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < K; ++j) {
      cd s = 0.0;
      for (int m = 0; m < M; ++m) s += W[k * M + m] * H[j * M + m];
      if (k == j) s -= t[k];
      E[k * K + j] = s;
    }
}

double fro2(int n, const cd* A) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += std::norm(A[i]);
  return s;
}

// G = H H^H  (K x K Hermitian)
void gram(int K, int M, const cd* H, cd* G) {
  for (int k = 0; k < K; ++k)
    for (int j = 0; j < K; ++j) {
      cd s = 0.0;
      for (int m = 0; m < M; ++m) s += H[k * M + m] * std::conj(H[j * M + m]);
      G[k * K + j] = s;
    }
}

// Lower Cholesky G = L L^H.  A pivot below 1e-12 times its diagonal entry of G
// counts as rank deficiency (H has rank < K): returns ORC_SINGULAR.
int cholesky(int K, const cd* G, cd* L) {
  for (int i = 0; i < K * K; ++i) L[i] = 0.0;
  for (int j = 0; j < K; ++j) {
    double d = G[j * K + j].real();
    for (int p = 0; p < j; ++p) d -= std::norm(L[j * K + p]);
    if (!(d > 1e-12 * G[j * K + j].real())) return ORC_SINGULAR;
    const double ljj = std::sqrt(d);
    L[j * K + j] = ljj;
    for (int i = j + 1; i < K; ++i) {
      cd s = G[i * K + j];
      for (int p = 0; p < j; ++p) s -= L[i * K + p] * std::conj(L[j * K + p]);
      L[i * K + j] = s / ljj;
    }
  }
  return ORC_OK;
}

// Solve G x = b with G = L L^H (forward then backward substitution).
void chol_solve(int K, const cd* L, const cd* b, cd* x) {
  std::vector<cd> z(K);
  for (int i = 0; i < K; ++i) {
    cd s = b[i];
    for (int p = 0; p < i; ++p) s -= L[i * K + p] * z[p];
    z[i] = s / L[i * K + i];
  }
  for (int i = K - 1; i >= 0; --i) {
    cd s = z[i];
    for (int p = i + 1; p < K; ++p) s -= std::conj(L[p * K + i]) * x[p];
    x[i] = s / L[i * K + i];
  }
}

// Y = E G^{-T}:  Y G^T = E  <=>  G y_k^T = e_k^T for every row k.
void right_solve_GT(int K, const cd* L, const cd* E, cd* Y) {
  std::vector<cd> b(K), x(K);
  for (int k = 0; k < K; ++k) {
    for (int j = 0; j < K; ++j) b[j] = E[k * K + j];
    chol_solve(K, L, b.data(), x.data());
    for (int j = 0; j < K; ++j) Y[k * K + j] = x[j];
  }
}

// W <- W - Y H^*   (K x K times K x M)
void sub_times_Hconj(int K, int M, const cd* Y, const cd* H, double scale, cd* W) {
  for (int k = 0; k < K; ++k)
    for (int m = 0; m < M; ++m) {
      cd s = 0.0;
      for (int j = 0; j < K; ++j) s += Y[k * K + j] * std::conj(H[j * M + m]);
      W[k * M + m] -= scale * s;
    }
}

// Column-wise prox of tau*||.||_{2,1}: w_m <- (1 - tau/max(||w_m||, tau)) w_m.
void prox_l21(int K, int M, cd* W, double tau) {
  for (int m = 0; m < M; ++m) {
    double p = 0.0;
    for (int k = 0; k < K; ++k) p += std::norm(W[k * M + m]);
    const double r = std::sqrt(p);
    const double f = (r > tau) ? (1.0 - tau / r) : 0.0;
    for (int k = 0; k < K; ++k) W[k * M + m] *= f;
  }
}

// Orthogonal projection onto A = {W : H W^T = S} (w.r.t. Re<.,.>):
//   P_A(X) = X - Y H^*,  Y G^T = X H^T - S.
void project_affine(int K, int M, const cd* H, const double* t, const cd* L, cd* X) {
  std::vector<cd> E(K * K), Y(K * K);
  residual_matrix(K, M, X, H, t, E.data());
  right_solve_GT(K, L, E.data(), Y.data());
  sub_times_Hconj(K, M, Y.data(), H, 1.0, X);
}

// ZF precoder W = S G^{-T} H^*: column m of G^{-T} H^* is conj(G^{-1} h_m).
void zf(int K, int M, const cd* H, const double* t, const cd* L, cd* W) {
  std::vector<cd> b(K), x(K);
  for (int m = 0; m < M; ++m) {
    for (int k = 0; k < K; ++k) b[k] = H[k * M + m];
    chol_solve(K, L, b.data(), x.data());
    for (int k = 0; k < K; ++k) W[k * M + m] = t[k] * std::conj(x[k]);
  }
}

// --------------------------------------------------------------- O1 / O2 bodies

// One paper layer (Eq. unfoldednet): V = W - eta (W H^T - S) H^*, then prox with
// threshold lambda*eta.  E_out (K x K) receives W H^T - S of the input W.
void ufpgd_layer(int K, int M, const cd* H, const double* t, double eta, double lam, cd* W,
                 cd* E_out) {
  residual_matrix(K, M, W, H, t, E_out);
  sub_times_Hconj(K, M, E_out, H, eta, W);
  prox_l21(K, M, W, lam * eta);
}

int ufpgd_forward(int K, int M, const cd* H, const double* t, int T, const double* eta,
                  const double* lam, const cd* W0, cd* W, cd* trace) {
  const int n = K * M;
  if (W0)
    for (int i = 0; i < n; ++i) W[i] = W0[i];
  else
    for (int i = 0; i < n; ++i) W[i] = std::conj(H[i]);  // W^(0) = H^* (Sec. VI-C)
  if (trace) std::copy(W, W + n, trace);
  std::vector<cd> E(K * K);
  for (int l = 0; l < T; ++l) {
    ufpgd_layer(K, M, H, t, eta[l], lam[l], W, E.data());
    if (trace) std::copy(W, W + n, trace + (size_t)(l + 1) * n);
  }
  return ORC_OK;
}

int ufproj_forward(int K, int M, const cd* H, const double* t, int T, const double* mu, cd* W,
                   cd* trace) {
  const int n = K * M;
  std::vector<cd> G(K * K), L(K * K);
  gram(K, M, H, G.data());
  if (cholesky(K, G.data(), L.data()) != ORC_OK) {
    for (int i = 0; i < n; ++i) W[i] = 0.0;
    if (trace) std::fill(trace, trace + (size_t)(T + 1) * n, cd(0.0));
    return ORC_SINGULAR;
  }
  zf(K, M, H, t, L.data(), W);  // W^(0) = ZF = P_A(H^*)
  if (trace) std::copy(W, W + n, trace);
  for (int l = 0; l < T; ++l) {
    prox_l21(K, M, W, mu[l]);
    project_affine(K, M, H, t, L.data(), W);
    if (trace) std::copy(W, W + n, trace + (size_t)(l + 1) * n);
  }
  return ORC_OK;
}

}  // namespace

extern "C" {

// ------------------------------------------------------------------ O5 metrics

double orc_l21(int K, int M, const double* W) { return l21(K, M, as_c(W)); }

// ||H W^T - S||_F
double orc_residual_fro(int K, int M, const double* H, const double* t, const double* W) {
  std::vector<cd> E(K * K);
  residual_matrix(K, M, as_c(W), as_c(H), t, E.data());
  return std::sqrt(fro2(K * K, E.data()));
}

// E = W H^T - S written out (K x K complex)
void orc_residual_matrix(int K, int M, const double* H, const double* t, const double* W,
                         double* E) {
  residual_matrix(K, M, as_c(W), as_c(H), t, as_c(E));
}

// SINR_k = |[H W^T]_kk|^2 / (sum_{j != k} |[H W^T]_kj|^2 + sigma^2)   (Sec. VI-B)
void orc_sinr(int K, int M, const double* H, const double* W, double sigma, double* sinr) {
  const cd* h = as_c(H);
  const cd* w = as_c(W);
  for (int k = 0; k < K; ++k) {
    double sig = 0.0, intf = 0.0;
    for (int j = 0; j < K; ++j) {
      cd a = 0.0;  // [H W^T]_{k,j} = sum_m H[k][m] W[j][m]
      for (int m = 0; m < M; ++m) a += h[k * M + m] * w[j * M + m];
      if (j == k)
        sig = std::norm(a);
      else
        intf += std::norm(a);
    }
    sinr[k] = sig / (intf + sigma * sigma);
  }
}

// R_sum = sum_k log2(1 + SINR_k)   (Sec. VI-B)
double orc_sum_rate(int K, int M, const double* H, const double* W, double sigma) {
  std::vector<double> s(K);
  orc_sinr(K, M, H, W, sigma, s.data());
  double r = 0.0;
  for (int k = 0; k < K; ++k) r += std::log2(1.0 + s[k]);
  return r;
}

// Gram matrix and Cholesky factor (exposed for pins)
int orc_gram_cholesky(int K, int M, const double* H, double* G, double* L) {
  gram(K, M, as_c(H), as_c(G));
  return cholesky(K, as_c(G), as_c(L));
}

// ZF precoder S G^{-T} H^* (the minimum-||W||_F feasible point)
int orc_zf(int K, int M, const double* H, const double* t, double* W) {
  std::vector<cd> G(K * K), L(K * K);
  gram(K, M, as_c(H), G.data());
  if (cholesky(K, G.data(), L.data()) != ORC_OK) return ORC_SINGULAR;
  zf(K, M, as_c(H), t, L.data(), as_c(W));
  return ORC_OK;
}

// PCG = ||W_ZF||_{2,1} / ||W||_{2,1}   (Sec. VI-B, same alpha cancels)
double orc_pcg(int K, int M, const double* H, const double* t, const double* W) {
  std::vector<cd> Wz(K * M);
  if (orc_zf(K, M, H, t, reinterpret_cast<double*>(Wz.data())) != ORC_OK) return NAN;
  return l21(K, M, Wz.data()) / l21(K, M, as_c(W));
}

// Orthogonal projection onto {W : H W^T = S}, in place.
int orc_project(int K, int M, const double* H, const double* t, double* X) {
  std::vector<cd> G(K * K), L(K * K);
  gram(K, M, as_c(H), G.data());
  if (cholesky(K, G.data(), L.data()) != ORC_OK) return ORC_SINGULAR;
  project_affine(K, M, as_c(H), t, L.data(), as_c(X));
  return ORC_OK;
}

// prox of tau*||.||_{2,1}, in place.
void orc_prox_l21(int K, int M, double* W, double tau) { prox_l21(K, M, as_c(W), tau); }

// ------------------------------------------------------------------ O1 / O2

// O1: T layers of Eq. (unfoldednet) with per-layer eta[l], lam[l].  W0 == NULL
// starts from H^*.  trace (nullable) receives all T+1 iterates.
int orc_ufpgd_forward(int K, int M, const double* H, const double* t, int T, const double* eta,
                      const double* lam, const double* W0, double* W, double* trace) {
  if (K < 1 || M < 1 || T < 0) return ORC_EINVAL;
  return ufpgd_forward(K, M, as_c(H), t, T, eta, lam, W0 ? as_c(W0) : nullptr, as_c(W),
                       trace ? as_c(trace) : nullptr);
}

// O2: T projected layers with per-layer shrink mu[l], from the ZF point.
int orc_ufproj_forward(int K, int M, const double* H, const double* t, int T, const double* mu,
                       double* W, double* trace) {
  if (K < 1 || M < 1 || T < 0) return ORC_EINVAL;
  return ufproj_forward(K, M, as_c(H), t, T, mu, as_c(W), trace ? as_c(trace) : nullptr);
}

// ------------------------------------------------------------------ O3: ADMM

// Long-run solve of  min ||W||_{2,1}  s.t.  H W^T = S  (Eq. optim1), by scaled
// ADMM on the split W = Z with W in A = {H W^T = S} and Z free:
//   W <- P_A(Z - U);  Z <- prox_{1/rho}(W + U);  U <- U + W - Z.
// rho follows residual balancing (factor 2 when one residual is 10x the other;
// U is rescaled with it).  Stops when ||W - Z||_F <= tol*max(||W||,||Z||) and
// rho*||Z - Z_prev||_F <= tol*rho*||U||_F, or after max_iter iterations.
// On return W is feasible, Z has exact zero columns, U is the scaled dual and
// *rho_io the final rho, so rho*U is a subgradient of ||.||_{2,1} at Z.
int orc_admm_solve(int K, int M, const double* H, const double* t, double* rho_io,
                   long max_iter, double tol, double* W_out, double* Z_out, double* U_out,
                   long* iters_out) {
  const int n = K * M;
  const cd* h = as_c(H);
  std::vector<cd> G(K * K), L(K * K);
  gram(K, M, h, G.data());
  if (cholesky(K, G.data(), L.data()) != ORC_OK) return ORC_SINGULAR;
  std::vector<cd> W(n), Z(n), U(n), Zp(n);
  zf(K, M, h, t, L.data(), Z.data());  // start from the ZF point, U = 0
  double rho = *rho_io;
  long it = 0;
  for (; it < max_iter; ++it) {
    for (int i = 0; i < n; ++i) W[i] = Z[i] - U[i];
    project_affine(K, M, h, t, L.data(), W.data());
    Zp = Z;
    for (int i = 0; i < n; ++i) Z[i] = W[i] + U[i];
    prox_l21(K, M, Z.data(), 1.0 / rho);
    for (int i = 0; i < n; ++i) U[i] += W[i] - Z[i];
    double r2 = 0.0, s2 = 0.0;
    for (int i = 0; i < n; ++i) {
      r2 += std::norm(W[i] - Z[i]);
      s2 += std::norm(Z[i] - Zp[i]);
    }
    const double r = std::sqrt(r2), s = rho * std::sqrt(s2);
    const double wn = std::sqrt(fro2(n, W.data())), zn = std::sqrt(fro2(n, Z.data()));
    const double un = rho * std::sqrt(fro2(n, U.data()));
    if (r <= tol * std::max(wn, zn) && s <= tol * un && it > 10) {
      ++it;
      break;
    }
    if (it % 20 == 19) {
      if (r > 10.0 * s) {
        rho *= 2.0;
        for (int i = 0; i < n; ++i) U[i] *= 0.5;
      } else if (s > 10.0 * r) {
        rho *= 0.5;
        for (int i = 0; i < n; ++i) U[i] *= 2.0;
      }
    }
  }
  std::copy(W.begin(), W.end(), as_c(W_out));
  if (Z_out) std::copy(Z.begin(), Z.end(), as_c(Z_out));
  if (U_out) std::copy(U.begin(), U.end(), as_c(U_out));
  *rho_io = rho;
  if (iters_out) *iters_out = it;
  return ORC_OK;
}

// ------------------------------------------------------------------ O4: long-run PGD

// Largest eigenvalue of G = H H^H (power iteration, FP64, to relative change 1e-15).
double orc_lambda_max(int K, int M, const double* H) {
  std::vector<cd> G(K * K), v(K, cd(1.0, 0.0)), w(K);
  gram(K, M, as_c(H), G.data());
  // deterministic non-degenerate start
  for (int k = 0; k < K; ++k) v[k] = cd(1.0 + 0.1 * k, 0.05 * k);
  double lam = 0.0;
  for (int it = 0; it < 100000; ++it) {
    for (int i = 0; i < K; ++i) {
      cd s = 0.0;
      for (int j = 0; j < K; ++j) s += G[i * K + j] * v[j];
      w[i] = s;
    }
    double nw = std::sqrt(fro2(K, w.data()));
    if (nw == 0.0) return 0.0;
    for (int i = 0; i < K; ++i) v[i] = w[i] / nw;
    if (std::fabs(nw - lam) <= 1e-15 * nw && it > 50) {
      lam = nw;
      break;
    }
    lam = nw;
  }
  return lam;
}

// PGD of Eq. (proxgd) with constant eta and lambda from W0 (NULL: H^*) until
// ||W_{k+1} - W_k||_F <= tol*max(1,||W_k||_F) or max_iter.  Its fixed point
// minimises F_P(W) = 2*lambda*||W||_{2,1} + ||H W^T - S||_F^2.
int orc_pgd_longrun(int K, int M, const double* H, const double* t, double eta, double lam,
                    long max_iter, double tol, const double* W0, double* W_out,
                    long* iters_out) {
  const int n = K * M;
  const cd* h = as_c(H);
  std::vector<cd> W(n), Wp(n), E(K * K);
  for (int i = 0; i < n; ++i) W[i] = W0 ? as_c(W0)[i] : std::conj(h[i]);
  long it = 0;
  for (; it < max_iter; ++it) {
    Wp = W;
    ufpgd_layer(K, M, h, t, eta, lam, W.data(), E.data());
    double d2 = 0.0;
    for (int i = 0; i < n; ++i) d2 += std::norm(W[i] - Wp[i]);
    if (std::sqrt(d2) <= tol * std::max(1.0, std::sqrt(fro2(n, Wp.data())))) {
      ++it;
      break;
    }
  }
  std::copy(W.begin(), W.end(), as_c(W_out));
  if (iters_out) *iters_out = it;
  return ORC_OK;
}

// F_P(W) = 2*lambda*||W||_{2,1} + ||H W^T - S||_F^2
double orc_penalised_objective(int K, int M, const double* H, const double* t, double lam,
                               const double* W) {
  std::vector<cd> E(K * K);
  residual_matrix(K, M, as_c(W), as_c(H), t, E.data());
  return 2.0 * lam * l21(K, M, as_c(W)) + fro2(K * K, E.data());
}

// ------------------------------------------------------------------ O6: gradients

// Unsupervised loss of Sec. V with weight a on the l2,1 term:
//   loss(W_T) = a*||W_T||_{2,1} + ||H W_T^T - S||_F^2.
// Supervised loss of Sec. V (the MSE to a ground-truth precoder W_gt):
//   loss(W_T) = ||W_T - W_gt||_F^2.
// Gradients are w.r.t. real parameters; a complex gradient G_W stands for
// dloss/dRe(W) + i dloss/dIm(W), with inner product <A,B> = Re sum conj(A) B.

namespace {

// dloss/dW at the output.  Unsupervised (Wgt == nullptr): a*w_m/||w_m|| (0 on zero
// columns) + 2 (W H^T - S) H^*.  Supervised: 2 (W - W_gt).
void loss_and_grad(int K, int M, const cd* H, const double* t, double a, const cd* W,
                   double* loss, cd* G, const cd* Wgt = nullptr) {
  if (Wgt) {
    double s = 0.0;
    for (int i = 0; i < K * M; ++i) {
      const cd d = W[i] - Wgt[i];
      s += std::norm(d);
      G[i] = 2.0 * d;
    }
    *loss = s;
    return;
  }
  std::vector<cd> E(K * K);
  residual_matrix(K, M, W, H, t, E.data());
  *loss = a * l21(K, M, W) + fro2(K * K, E.data());
  for (int k = 0; k < K; ++k)
    for (int m = 0; m < M; ++m) {
      cd s = 0.0;
      for (int j = 0; j < K; ++j) s += E[k * K + j] * std::conj(H[j * M + m]);
      G[k * M + m] = 2.0 * s;
    }
  for (int m = 0; m < M; ++m) {
    double p = 0.0;
    for (int k = 0; k < K; ++k) p += std::norm(W[k * M + m]);
    const double r = std::sqrt(p);
    if (r > 0.0)
      for (int k = 0; k < K; ++k) G[k * M + m] += a * W[k * M + m] / r;
  }
}

// Reverse through x_m = (1 - tau/r) v_m (r = ||v_m|| > tau; else x_m = 0):
// G <- (1 - tau/r) G + (tau/r^3) Re(v^H G) v on active columns, 0 elsewhere;
// returns dloss/dtau = -sum_active Re(v^H G)/r.
double shrink_backward(int K, int M, const cd* V, double tau, cd* G) {
  double dtau = 0.0;
  for (int m = 0; m < M; ++m) {
    double p = 0.0;
    for (int k = 0; k < K; ++k) p += std::norm(V[k * M + m]);
    const double r = std::sqrt(p);
    if (r > tau) {
      double vg = 0.0;  // Re(v^H g)
      for (int k = 0; k < K; ++k) vg += (std::conj(V[k * M + m]) * G[k * M + m]).real();
      dtau -= vg / r;
      const double c1 = 1.0 - tau / r, c2 = tau / (r * r * r) * vg;
      for (int k = 0; k < K; ++k) G[k * M + m] = c1 * G[k * M + m] + c2 * V[k * M + m];
    } else {
      for (int k = 0; k < K; ++k) G[k * M + m] = 0.0;
    }
  }
  return dtau;
}

}  // namespace

// Gradient of the loss after T projected layers w.r.t. mu[0..T-1].
// The projection X -> P_A(X) is affine with a self-adjoint linear part
// X -> X - (X H^T) G^{-T} H^*, so its adjoint applies that same map.
// Wgt (K x M complex, or NULL): the supervised loss's label; NULL selects the
// unsupervised loss with weight a.
int orc_ufproj_grad_loss(int K, int M, const double* H, const double* t, int T, const double* mu,
                         double a, const double* Wgt, double* loss, double* dmu) {
  const int n = K * M;
  const cd* h = as_c(H);
  std::vector<cd> trace((size_t)(T + 1) * n);
  std::vector<cd> W(n);
  int st = ufproj_forward(K, M, h, t, T, mu, W.data(), trace.data());
  if (st != ORC_OK) return st;
  std::vector<cd> Gm(K * K), L(K * K);
  gram(K, M, h, Gm.data());
  cholesky(K, Gm.data(), L.data());
  std::vector<cd> g(n), E(K * K), Y(K * K);
  loss_and_grad(K, M, h, t, a, W.data(), loss, g.data(), Wgt ? as_c(Wgt) : nullptr);
  std::vector<double> zeros(K, 0.0);
  for (int l = T - 1; l >= 0; --l) {
    // through the linear part of the projection: g <- g - (g H^T) G^{-T} H^*
    residual_matrix(K, M, g.data(), h, zeros.data(), E.data());
    right_solve_GT(K, L.data(), E.data(), Y.data());
    sub_times_Hconj(K, M, Y.data(), h, 1.0, g.data());
    // through the shrink of layer l (its input is iterate l)
    dmu[l] = shrink_backward(K, M, trace.data() + (size_t)l * n, mu[l], g.data());
  }
  return ORC_OK;
}

int orc_ufproj_grad(int K, int M, const double* H, const double* t, int T, const double* mu,
                    double a, double* loss, double* dmu) {
  return orc_ufproj_grad_loss(K, M, H, t, T, mu, a, nullptr, loss, dmu);
}

// Gradient of the loss after T paper layers w.r.t. eta[] and lam[] (W^(0) = H^*);
// Wgt as for orc_ufproj_grad_loss.
int orc_ufpgd_grad_loss(int K, int M, const double* H, const double* t, int T, const double* eta,
                        const double* lam, double a, const double* Wgt, double* loss,
                        double* deta, double* dlam) {
  const int n = K * M;
  const cd* h = as_c(H);
  std::vector<cd> trace((size_t)(T + 1) * n), W(n);
  ufpgd_forward(K, M, h, t, T, eta, lam, nullptr, W.data(), trace.data());
  std::vector<cd> g(n), E(K * K), V(n), EH(n), GE(K * K);
  std::vector<double> zeros(K, 0.0);
  loss_and_grad(K, M, h, t, a, W.data(), loss, g.data(), Wgt ? as_c(Wgt) : nullptr);
  for (int l = T - 1; l >= 0; --l) {
    const cd* Win = trace.data() + (size_t)l * n;
    // recompute V = W - eta E H^* and EH = E H^*
    residual_matrix(K, M, Win, h, t, E.data());
    for (int i = 0; i < n; ++i) EH[i] = 0.0;
    sub_times_Hconj(K, M, E.data(), h, -1.0, EH.data());  // EH = + E H^*
    for (int i = 0; i < n; ++i) V[i] = Win[i] - eta[l] * EH[i];
    const double dtau = shrink_backward(K, M, V.data(), lam[l] * eta[l], g.data());
    double gv_eh = 0.0;  // <g_V, E H^*>
    for (int i = 0; i < n; ++i) gv_eh += (std::conj(g[i]) * EH[i]).real();
    deta[l] = -gv_eh + lam[l] * dtau;
    dlam[l] = eta[l] * dtau;
    // through V = W (I - eta H^T H^*): g <- g - eta (g H^T) H^*
    residual_matrix(K, M, g.data(), h, zeros.data(), GE.data());
    sub_times_Hconj(K, M, GE.data(), h, eta[l], g.data());
  }
  return ORC_OK;
}

int orc_ufpgd_grad(int K, int M, const double* H, const double* t, int T, const double* eta,
                   const double* lam, double a, double* loss, double* deta, double* dlam) {
  return orc_ufpgd_grad_loss(K, M, H, t, T, eta, lam, a, nullptr, loss, deta, dlam);
}

// ------------------------------------------------------------------ batch harness

// Runs O1 (mode 0) or O2 (mode 1) independently on B instances, splitting
// [0, B) into nthreads contiguous ranges.  H: [B][K][M] complex, t: [B][K],
// p1 = eta (mode 0) or mu (mode 1), p2 = lam (mode 0, else unused).
// Per instance: W, obj = ||W||_{2,1}, resid = ||H W^T - S||_F, status.
int orc_batch_forward(int mode, int nthreads, long B, int K, int M, const double* H,
                      const double* t, int T, const double* p1, const double* p2, double* W,
                      double* obj, double* resid, int* status) {
  if (nthreads < 1) nthreads = 1;
  const long n = (long)K * M;
  auto work = [&](long b0, long b1) {
    for (long b = b0; b < b1; ++b) {
      const double* Hb = H + 2 * n * b;
      const double* tb = t + (long)K * b;
      double* Wb = W + 2 * n * b;
      int st = (mode == 0) ? orc_ufpgd_forward(K, M, Hb, tb, T, p1, p2, nullptr, Wb, nullptr)
                           : orc_ufproj_forward(K, M, Hb, tb, T, p1, Wb, nullptr);
      if (status) status[b] = st;
      if (obj) obj[b] = orc_l21(K, M, Wb);
      if (resid) resid[b] = orc_residual_fro(K, M, Hb, tb, Wb);
    }
  };
  std::vector<std::thread> th;
  const long per = (B + nthreads - 1) / nthreads;
  for (int i = 0; i < nthreads; ++i) {
    long b0 = i * per, b1 = std::min(B, b0 + per);
    if (b0 >= b1) break;
    th.emplace_back(work, b0, b1);
  }
  for (auto& x : th) x.join();
  return ORC_OK;
}

// Same split for the ADMM solve (used for optimality-gap statistics).
int orc_batch_admm(int nthreads, long B, int K, int M, const double* H, const double* t,
                   double rho, long max_iter, double tol, double* W, long* iters, int* status) {
  if (nthreads < 1) nthreads = 1;
  const long n = (long)K * M;
  auto work = [&](long b0, long b1) {
    for (long b = b0; b < b1; ++b) {
      double r = rho;
      long it = 0;
      int st = orc_admm_solve(K, M, H + 2 * n * b, t + (long)K * b, &r, max_iter, tol,
                              W + 2 * n * b, nullptr, nullptr, &it);
      if (iters) iters[b] = it;
      if (status) status[b] = st;
    }
  };
  std::vector<std::thread> th;
  const long per = (B + nthreads - 1) / nthreads;
  for (int i = 0; i < nthreads; ++i) {
    long b0 = i * per, b1 = std::min(B, b0 + per);
    if (b0 >= b1) break;
    th.emplace_back(work, b0, b1);
  }
  for (auto& x : th) x.join();
  return ORC_OK;
}

}  // extern "C"
