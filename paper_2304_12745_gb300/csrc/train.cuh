// Forward + reverse (adjoint) pass of T unfolded layers per instance, for
// learning the per-layer parameters (Sec. V, learning rule).  Loss per instance:
// the unsupervised cost  a ||W_T||_{2,1} + ||H W_T^T - S||_F^2, or with labels
// (TrainArgs::wgt) the supervised cost  ||W_T - W_gt||_F^2.
//
// Gradients are taken w.r.t. real parameters; a complex gradient g stands for
// dloss/dRe(W) + i dloss/dIm(W) with <A, B> = Re sum conj(A) B.  Reverse rules:
//   output:     g = a w_m/||w_m|| (non-zero columns) + 2 (W H^T - S) H^*
//               (supervised: g = 2 (W - W_gt))
//   projection: W = X - (X H^T - S) Q has the self-adjoint linear part
//               X -> X - (X H^T) Q, so g <- g - (g H^T) Q
//   paper step: V = W - eta (W H^T - S) H^* has the self-adjoint linear part
//               W -> W - eta (W H^T) H^*, so g <- g - eta (g H^T) H^*, and
//               dloss/deta += -<(g_V H^T), E>
//   shrink:     x = (1 - tau/r) v (r = ||v|| > tau, else 0):
//               g <- (1 - tau/r) g + (tau/r^3) Re(v^H g) v on active columns, 0 else,
//               dloss/dtau = -sum_active Re(v^H g)/r
// Memory: instead of storing every W_t, the forward pass keeps W at every c-th
// layer (c = ceil(sqrt(T))) in workspace and the reverse pass recomputes W_{l}
// from the nearest checkpoint before undoing layer l.
#pragma once

#include "solve.cuh"

namespace precode {

struct TrainArgs {
  SolveArgs s;      // H, t, t_stride, step, lam, B, K, M, T, cond_thr, opts, err, flags
  float a;          // weight of ||W_T||_{2,1} in the unsupervised loss
  const float2* wgt;  // supervised loss: labels W_gt [B][K][M] (W's layout), else nullptr
  float2* cp;       // checkpoints [B][ncp][KB*MB] (bucket-sized slots); nullptr: in
                    // tensor memory (kernels that keep ncp of them on chip)
  int cp_every;     // checkpoint interval c
  int ncp;          // checkpoints per instance = ceil(T / c)
  float* part;      // per-instance [B][1 + 2T]: loss, d step[T], d lam[T]
};

template <int MODE, int KB, int MB, int GK, int GM, int JC_, bool EXACT, int NW>
struct TrainKernel : SolveKernel<MODE, KB, MB, GK, GM, JC_, EXACT, NW, true, false> {
  using Base = SolveKernel<MODE, KB, MB, GK, GM, JC_, EXACT, NW, true, false>;
  using C = typename Base::C;
  using Ctx = typename Base::Ctx;
  using WReg = typename Base::WReg;
  using EReg = typename Base::EReg;
  using CT = typename Base::CT;
  static constexpr int TPI = C::TPI, UPT = C::UPT, PPT = C::PPT, NA = C::NA, NJC = C::NJC,
                       WPG = C::WPG, LPW = C::LPW;
  static constexpr int ES2_BYTES = KB * KB * 8;
  static constexpr int GROUP_STRIDE = align_up(C::GROUP_BYTES + ES2_BYTES, 16);
  static constexpr int SMEM_BYTES = C::GROUPS * GROUP_STRIDE;

  // sum of x over the whole instance group (identical result in every thread)
  __device__ __forceinline__ static float group_sum(const Ctx& c, float x) {
#pragma unroll
    for (int msk = 1; msk < LPW; msk <<= 1) x += __shfl_xor_sync(c.wmask, x, msk);
    if constexpr (WPG > 1) {
      Base::gsync(c);
      if (c.lane == 0) c.wsum[c.wig] = x;
      Base::gsync(c);
      x = 0.f;
      for (int ww = 0; ww < WPG; ++ww) x += c.wsum[ww];
    }
    return x;
  }

  // per-antenna sums over all users of the column (like the column norms)
  __device__ __forceinline__ static void col_allreduce(const Ctx& c, float (&v)[NA]) {
#pragma unroll
    for (int msk = GM; msk < LPW; msk <<= 1)
#pragma unroll
      for (int q = 0; q < NA; ++q) v[q] += __shfl_xor_sync(c.wmask, v[q], msk);
    if constexpr (WPG > 1) {
      float* buf = c.nrm;
      if (c.lane < GM)
#pragma unroll
        for (int q = 0; q < NA; ++q) buf[(c.wig * GM + c.b) * NA + q] = v[q];
      Base::gsync(c);
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        float s = 0.f;
        for (int ww = 0; ww < WPG; ++ww) s += buf[(ww * GM + c.b) * NA + q];
        v[q] = s;
      }
      Base::gsync(c);
    }
  }

  // w -= scale * Es[k_u][:] * X  (CJ: X conjugated)
  template <bool CJ>
  __device__ __forceinline__ static void update_s(const Ctx& c, WReg& w, const float2* X,
                                                  float scale) {
    const int K = Base::Kd(c), M = Base::Md(c);
#pragma unroll 2
    for (int j = 0; j < KB; ++j) {
      if (!EXACT && j >= K) break;
      float2 ej[UPT];
#pragma unroll
      for (int u = 0; u < UPT; ++u) {
        const float2 v = c.Es[Base::user(c, u) * KB + j];
        ej[u] = make_float2(v.x * scale, v.y * scale);
      }
      const float2* row = X + j * M;
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        if (!Base::pok(c, i)) continue;
        const float4 v = *reinterpret_cast<const float4*>(row + 2 * Base::pair(c, i));
        const float2 x0 = make_float2(v.x, v.y), x1 = make_float2(v.z, v.w);
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          if (CJ) {
            cmsub_conj(w[u][2 * i], ej[u], x0);
            cmsub_conj(w[u][2 * i + 1], ej[u], x1);
          } else {
            cmsub(w[u][2 * i], ej[u], x0);
            cmsub(w[u][2 * i + 1], ej[u], x1);
          }
        }
      }
    }
  }

  // Es <- X H^T (minus S, times scale) for the rows held in x
  __device__ __forceinline__ static float residual(const Ctx& c, const WReg& x, EReg& e,
                                                   float scale, bool sub_s) {
    float rs = 0.f;
#pragma unroll 1
    for (int jc = 0; jc < NJC; ++jc) {
      Base::partials(c, x, c.Hs, jc, e);
      rs += Base::reduce(c, e, jc, scale, sub_s);
    }
    Base::gsync(c);  // Es complete for every row group
    return rs;
  }

  // one forward layer l (W_l -> W_{l+1})
  __device__ __forceinline__ static void fwd_layer(const Ctx& c, const TrainArgs& A, WReg& w,
                                                   EReg& e, float (&r2)[NA], int l, float invL) {
    if constexpr (MODE == kModeProj) {
      Base::colnorm2(c, w, r2);
      Base::shrink(w, r2, fmaxf(__ldg(A.s.step + l), 0.f));
      residual(c, w, e, 1.f, true);
      Base::template update<false>(c, w, c.Qs);
    } else {
      const float eta = __ldg(A.s.step + l) * invL;
      residual(c, w, e, eta, true);
      Base::template update<true>(c, w, c.Hs);
      Base::colnorm2(c, w, r2);
      Base::shrink(w, r2, fmaxf(fmaxf(__ldg(A.s.lam + l), 0.f) * eta, 0.f));
    }
  }

  __device__ __forceinline__ static float2* cp_slot(const TrainArgs& A, int64_t inst, int k) {
    return A.cp + ((size_t)inst * A.ncp + k) * (size_t)(KB * MB);
  }

  __device__ __forceinline__ static void store_cp(const Ctx& c, const TrainArgs& A, int64_t inst,
                                                  int k, const WReg& w) {
    float2* dst = cp_slot(A, inst, k);
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int i = 0; i < PPT; ++i)
        *reinterpret_cast<float4*>(dst + Base::user(c, u) * MB + 2 * Base::pair(c, i)) =
            make_float4(w[u][2 * i].x, w[u][2 * i].y, w[u][2 * i + 1].x, w[u][2 * i + 1].y);
  }

  __device__ __forceinline__ static void load_cp(const Ctx& c, const TrainArgs& A, int64_t inst,
                                                 int k, WReg& w) {
    const float2* src = cp_slot(A, inst, k);
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        const float4 v =
            *reinterpret_cast<const float4*>(src + Base::user(c, u) * MB + 2 * Base::pair(c, i));
        w[u][2 * i] = mkc<CT>(v.x, v.y);
        w[u][2 * i + 1] = mkc<CT>(v.z, v.w);
      }
  }

  // reverse through the group shrink at input v (threshold tau): g in place.
  // Returns dloss/dtau (identical in every thread).
  __device__ __forceinline__ static float shrink_back(const Ctx& c, const WReg& v, WReg& g,
                                                      const float (&r2)[NA], float tau) {
    float vg[NA];
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      float s = 0.f;
#pragma unroll
      for (int u = 0; u < UPT; ++u) s = fmaf(v[u][q].x, g[u][q].x, fmaf(v[u][q].y, g[u][q].y, s));
      vg[q] = s;
    }
    col_allreduce(c, vg);
    float dtau = 0.f;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const bool act = r2[q] > tau * tau && r2[q] > 0.f;
      const float ir = act ? rsqrtf(r2[q]) : 0.f;
      const float c1 = act ? 1.f - tau * ir : 0.f;
      const float c2 = act ? tau * ir * ir * ir * vg[q] : 0.f;
      dtau -= act ? vg[q] * ir : 0.f;
#pragma unroll
      for (int u = 0; u < UPT; ++u) {
        g[u][q].x = c1 * g[u][q].x + c2 * v[u][q].x;
        g[u][q].y = c1 * g[u][q].y + c2 * v[u][q].y;
      }
    }
    // antennas are spread over the GM threads of a row; every row holds the same sums
#pragma unroll
    for (int msk = 1; msk < GM; msk <<= 1) dtau += __shfl_xor_sync(c.wmask, dtau, msk);
    return dtau;
  }

  __device__ static void run(const TrainArgs& A) {
    extern __shared__ __align__(16) unsigned char smem[];
    Ctx c;
    const int tid = threadIdx.x;
    c.gid = tid / TPI;
    c.g = tid - c.gid * TPI;
    c.b = c.g % GM;
    c.a = c.g / GM;
    c.lane = tid & 31;
    c.wig = c.g >> 5;
    c.wmask = TPI >= 32 ? 0xffffffffu : (((1u << (TPI & 31)) - 1u) << ((c.lane / TPI) * TPI));
    unsigned char* gs = smem + c.gid * GROUP_STRIDE;
    c.Hs = reinterpret_cast<float2*>(gs + C::H_OFF);
    c.Qs = reinterpret_cast<float2*>(gs + C::Q_OFF);
    c.red = reinterpret_cast<float*>(gs + C::RED_OFF);
    c.Es = reinterpret_cast<float2*>(gs + C::E_OFF);
    c.nrm = reinterpret_cast<float*>(gs + C::NRM_OFF);
    c.tks = reinterpret_cast<float*>(gs + C::SC_OFF);
    c.dsc = c.tks + KB;
    c.piv = c.dsc + KB;
    c.misc = reinterpret_cast<int*>(c.piv + KB);
    c.wsum = reinterpret_cast<float*>(c.misc + 8);
    c.bar = reinterpret_cast<uint64_t*>(gs + C::BAR_OFF);
    float2* Es2 = reinterpret_cast<float2*>(gs + C::GROUP_BYTES);
    if (c.g == 0) mbar_init(c.bar, 1);
    fence_mbar_init();
    __syncthreads();

    const int T = A.s.T;
    const int PW = 1 + 2 * T;
    uint32_t phase = 0;
    WReg w, g;
    EReg e;
    float r2[NA];
#pragma unroll 1
    for (int64_t inst = (int64_t)blockIdx.x * C::GROUPS + c.gid; inst < A.s.B;
         inst += (int64_t)gridDim.x * C::GROUPS) {
      c.K = A.s.K;
      c.M = A.s.M;
      const int K = Base::Kd(c), M = Base::Md(c);
      const int64_t h_off = inst * (int64_t)A.s.K * A.s.M;
      const int64_t t_off = inst * A.s.t_stride;
      float* part = A.part + inst * PW;

      gsync_all(c);
      if (c.g == 0 && !(A.s.opts & OPT_STALL_COPY)) {
        fence_proxy_async_smem();
        const uint32_t bytes = (uint32_t)(K * M) * 8u;
        mbar_arrive_expect_tx(c.bar, bytes);
        bulk_g2s(c.Hs, A.s.H + h_off, bytes, c.bar);
      }
      if (c.g < K) c.tks[c.g] = A.s.t[t_off + c.g];
      if (c.g == 0) c.misc[0] = mbar_wait_bounded(c.bar, phase, copy_wait_ns(A.s)) ? 1 : 0;
      Base::gsync(c);
      if (c.misc[0] == 0) {
        if (c.g == 0) {
          atomicAdd(A.s.err, 1ull);
          if (A.s.flags) A.s.flags[inst] = PRECODE_F_TIMEOUT;
          c.misc[1] = mbar_wait_bounded(c.bar, phase, copy_wait_ns(A.s)) ? 1 : 0;
        }
        Base::gsync(c);
        for (int j = c.g; j < PW; j += TPI) part[j] = 0.f;
        if (c.misc[1] == 0) return;
        phase ^= 1;
        continue;
      }
      if (c.g != 0) mbar_wait_bounded(c.bar, phase, copy_wait_ns(A.s));
      phase ^= 1;

      // ---- setup: W^(0)
      int fl = 0;
      float invL = 1.f;
      Base::load_rows(c, w, c.Hs);
#pragma unroll
      for (int u = 0; u < UPT; ++u)
#pragma unroll
        for (int q = 0; q < NA; ++q) w[u][q].y = -w[u][q].y;  // conj(H) rows
      if (MODE == kModeProj || (A.s.opts & OPT_STEP_NORMALISED)) {
        residual(c, w, e, 1.f, false);  // Es = G^T
        if constexpr (MODE == kModeProj) {
          fl = Base::setup_proj(c, w, A.s.cond_thr);
        } else {
          invL = Base::inv_gershgorin(c);
        }
      }
      if (fl & PRECODE_F_SINGULAR) {  // W_T = 0: ||S||_F^2, or ||W_gt||_F^2 with labels
        float s2 = 0.f;
        if (A.wgt) {
          for (int idx = c.g; idx < K * M; idx += TPI) {
            const float2 lb = A.wgt[h_off + idx];
            s2 += lb.x * lb.x + lb.y * lb.y;
          }
          s2 = group_sum(c, s2);
        } else {
          for (int k = 0; k < K; ++k) s2 += c.tks[k] * c.tks[k];
        }
        for (int j = c.g; j < PW; j += TPI) part[j] = (j == 0) ? s2 : 0.f;
        if (c.g == 0 && A.s.flags) A.s.flags[inst] = fl;
        continue;
      }

      // ---- forward with checkpoints
#pragma unroll 1
      for (int l = 0; l < T; ++l) {
        if (l % A.cp_every == 0) store_cp(c, A, inst, l / A.cp_every, w);
        fwd_layer(c, A, w, e, r2, l, invL);
      }

      // ---- loss and its gradient at W_T
      if (A.wgt) {  // supervised: ||W_T - W_gt||_F^2, g = 2 (W_T - W_gt)
        float s2 = 0.f;
#pragma unroll
        for (int u = 0; u < UPT; ++u)
#pragma unroll
          for (int i = 0; i < PPT; ++i) {
            float4 lb = make_float4(0.f, 0.f, 0.f, 0.f);
            if (Base::uok(c, u) && Base::pok(c, i))
              lb = *reinterpret_cast<const float4*>(A.wgt + h_off + (int64_t)Base::user(c, u) * M +
                                                   2 * Base::pair(c, i));
            else
              lb = make_float4(w[u][2 * i].x, w[u][2 * i].y, w[u][2 * i + 1].x, w[u][2 * i + 1].y);
            const float d0 = w[u][2 * i].x - lb.x, d1 = w[u][2 * i].y - lb.y;
            const float d2 = w[u][2 * i + 1].x - lb.z, d3 = w[u][2 * i + 1].y - lb.w;
            s2 += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
            g[u][2 * i] = mkc<CT>(2.f * d0, 2.f * d1);
            g[u][2 * i + 1] = mkc<CT>(2.f * d2, 2.f * d3);
          }
        const float lsum = group_sum(c, s2);
        if (c.g == 0) part[0] = lsum;
      } else {
      Base::colnorm2(c, w, r2);
      float o = 0.f;
#pragma unroll
      for (int q = 0; q < NA; ++q) o += sqrtf(r2[q]);
#pragma unroll
      for (int msk = 1; msk < GM; msk <<= 1) o += __shfl_xor_sync(c.wmask, o, msk);
      const float rs = group_sum(c, residual(c, w, e, 1.f, true));
#pragma unroll
      for (int u = 0; u < UPT; ++u)
#pragma unroll
        for (int q = 0; q < NA; ++q) g[u][q] = mkc<CT>(0.f, 0.f);
      update_s<true>(c, g, c.Hs, -2.f);  // g = 2 E_T H^*
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        const float ir = r2[q] > 0.f ? A.a * rsqrtf(r2[q]) : 0.f;
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          g[u][q].x = fmaf(ir, w[u][q].x, g[u][q].x);
          g[u][q].y = fmaf(ir, w[u][q].y, g[u][q].y);
        }
      }
      if (c.g == 0) part[0] = A.a * o + rs;
      }

      // ---- reverse: layer l = T-1 .. 0, recomputing its input from a checkpoint
#pragma unroll 1
      for (int l = T - 1; l >= 0; --l) {
        const int k = l / A.cp_every;
        Base::gsync(c);  // Es / red free before the recomputation reuses them
        load_cp(c, A, inst, k, w);
#pragma unroll 1
        for (int s = k * A.cp_every; s < l; ++s) fwd_layer(c, A, w, e, r2, s, invL);
        // w = W_l, the input of layer l
        if constexpr (MODE == kModeProj) {
          residual(c, g, e, 1.f, false);  // Es = g H^T
          update_s<false>(c, g, c.Qs, 1.f);  // g <- g - (g H^T) Q
          Base::colnorm2(c, w, r2);
          const float mu = fmaxf(__ldg(A.s.step + l), 0.f);
          const float dmu = shrink_back(c, w, g, r2, mu);
          if (c.g == 0) part[1 + l] = (__ldg(A.s.step + l) > 0.f) ? dmu : 0.f;
        } else {
          const float eta = __ldg(A.s.step + l) * invL;
          const float lam_raw = __ldg(A.s.lam + l);
          const float lam = fmaxf(lam_raw, 0.f);
          const float tau = fmaxf(lam * eta, 0.f);
          residual(c, w, e, 1.f, true);  // Es = E_l = W_l H^T - S
          for (int idx = c.g; idx < KB * KB; idx += TPI) Es2[idx] = c.Es[idx];
          update_s<true>(c, w, c.Hs, eta);  // w = V_l
          Base::colnorm2(c, w, r2);
          const float dtau = shrink_back(c, w, g, r2, tau);  // g = dloss/dV_l
          residual(c, g, e, 1.f, false);                       // Es = g_V H^T
          float dot = 0.f;
          for (int idx = c.g; idx < KB * KB; idx += TPI) {
            const float2 x = c.Es[idx], y = Es2[idx];
            dot = fmaf(x.x, y.x, fmaf(x.y, y.y, dot));
          }
          dot = group_sum(c, dot);
          update_s<true>(c, g, c.Hs, eta);  // g <- g_V - eta (g_V H^T) H^*
          const bool tau_on = lam * eta > 0.f;
          const float deta = -dot + (tau_on ? lam * dtau : 0.f);
          const float dlam = (tau_on && lam_raw > 0.f) ? eta * dtau : 0.f;
          if (c.g == 0) {
            part[1 + l] = deta * invL;
            part[1 + T + l] = dlam;
          }
        }
      }
      if (c.g == 0 && A.s.flags) A.s.flags[inst] = fl;
      if constexpr (MODE == kModeProj)
        for (int j = 1 + T + c.g; j < PW; j += TPI) part[j] = 0.f;
    }
  }

  __device__ __forceinline__ static void gsync_all(const Ctx& c) { Base::gsync(c); }
};

template <int MODE, int KB, int MB, int GK, int GM, int JC, bool EXACT, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) train_kernel(TrainArgs A) {
  TrainKernel<MODE, KB, MB, GK, GM, JC, EXACT, NW>::run(A);
}

}  // namespace precode
