// Forward + adjoint of T unfolded layers on the tensor cores, K = 8 users,
// M = 64 antennas, one warp per instance (the layout and building blocks of
// the K = 8 tensor-core solve kernel).  Loss per instance and reverse rules as
// in the FP32 training kernel:
//   loss        a ||W_T||_{2,1} + ||H W_T^T - S||_F^2
//   output      g = a w_m / ||w_m|| + 2 (W_T H^T - S) H^*
//   projection  g <- g - (g H^T) Q                      (self-adjoint linear part)
//   paper step  g <- g - eta (g H^T) H^*,  d eta += -<g_V H^T, E_l>
//   shrink      g <- (1 - tau/r) g + (tau/r^3) Re(v^H g) v on active columns, 0 else,
//               d tau = -sum_active Re(v^H g) / r
// All contractions, including g H^T and the updates of g, are split-TF32 warp
// MMAs.  W_l is kept at every c-th layer (c = ceil(sqrt(T))) in global memory,
// in the lane fragment order, and the reverse pass recomputes the layers in
// between.
#pragma once

#include "solve_tc.cuh"
#include "train.cuh"

namespace precode {

template <int MODE, int NW>
struct TrainTC {
  using S = SolveTC<MODE, NW, false>;
  using Base = typename S::Base;
  using C = typename S::C;
  using Ctx = typename S::Ctx;
  using Lane = typename S::Lane;
  using WT = typename S::WT;
  static constexpr int KB = 8, MB = 64;
  // per warp: the solve kernel's layout, a second shrink-factor buffer and (projected
  // layer) the raw conj(H) B fragments for the loss gradient's E_T H^*
  static constexpr int OFF_FB2 = S::GROUP_STRIDE;
  static constexpr int OFF_XR = OFF_FB2 + 256;
  static constexpr int GROUP_STRIDE = OFF_XR + (MODE == kModeProj ? 8 * 32 * 16 : 0);
  static constexpr int SMEM_BYTES = NW * GROUP_STRIDE;

  // column sums of Re(v^H g) over the 8 users, read out like S::colsum
  __device__ __forceinline__ static float2 colsum_vg(const Lane& L, float* nb, const WT& v,
                                                     const WT& g) {
    const int sw = S::nb_swz(L.lane);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float4 p;
      p.x = fmaf(v[2 * j][0], g[2 * j][0], v[2 * j][2] * g[2 * j][2]);
      p.y = fmaf(v[2 * j][1], g[2 * j][1], v[2 * j][3] * g[2 * j][3]);
      p.z = fmaf(v[2 * j + 1][0], g[2 * j + 1][0], v[2 * j + 1][2] * g[2 * j + 1][2]);
      p.w = fmaf(v[2 * j + 1][1], g[2 * j + 1][1], v[2 * j + 1][3] * g[2 * j + 1][3]);
      *reinterpret_cast<float4*>(nb + L.lane * 16 + 4 * (j ^ sw)) = p;
    }
    __syncwarp();
    const int rq = L.lane & 3, rs = L.lane >> 2;
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int gg = 0; gg < 8; ++gg) {
      const int wr = 4 * gg + rq;
      const float2 x = *reinterpret_cast<const float2*>(nb + wr * 16 + 4 * ((rs >> 1) ^ S::nb_swz(wr)) +
                                                       (rs & 1) * 2);
      a.x += x.x;
      a.y += x.y;
    }
    return a;
  }

  // factors (f0, f1) of the reading lane's two columns to fb; every lane then
  // gets its 16 columns' factors (as S::shrink distributes them)
  __device__ __forceinline__ static void put_factors(const Lane& L, float* fb, float f0, float f1) {
    const int rq = L.lane & 3, rs = L.lane >> 2;
    *reinterpret_cast<float2*>(fb + rq * 16 + 4 * ((rs >> 1) ^ (rq & 2)) + (rs & 1) * 2) =
        make_float2(f0, f1);
  }
  __device__ __forceinline__ static float4 get_factors(const Lane& L, const float* fb, int j) {
    return *reinterpret_cast<const float4*>(fb + L.q * 16 + 4 * (j ^ (L.q & 2)));
  }

  // Supervised loss of the lane's entries and its gradient, in original units:
  // W_T = f w (f: the output factor of the units w is held in), labels lb at
  // [K][M] (row g, antennas 8s + 2q + {0, 1}); g = 2 (W_T - W_gt).  Returns the
  // instance's ||W_T - W_gt||_F^2 (warp sum).
  __device__ __forceinline__ static float sup_loss_grad(const Lane& L, const float2* lb, float f,
                                                        const WT& w, WT& g) {
    float s2 = 0.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float4 v = *reinterpret_cast<const float4*>(lb + L.g * MB + 8 * s + 2 * L.q);
      const float d0 = f * w[s][0] - v.x, d1 = f * w[s][1] - v.z;
      const float d2 = f * w[s][2] - v.y, d3 = f * w[s][3] - v.w;
      s2 += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
      g[s][0] = 2.f * d0;
      g[s][1] = 2.f * d1;
      g[s][2] = 2.f * d2;
      g[s][3] = 2.f * d3;
    }
#pragma unroll
    for (int msk = 1; msk < 32; msk <<= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, msk);
    return s2;
  }
  // ||W_gt||_F^2 of one instance's labels (warp sum).
  __device__ __forceinline__ static float sup_loss_zero(const Lane& L, const float2* lb) {
    float s2 = 0.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float4 v = *reinterpret_cast<const float4*>(lb + L.g * MB + 8 * s + 2 * L.q);
      s2 += v.x * v.x + v.y * v.y + v.z * v.z + v.w * v.w;
    }
#pragma unroll
    for (int msk = 1; msk < 32; msk <<= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, msk);
    return s2;
  }

  // g <- d loss / d v through the group shrink with threshold tau at input v;
  // returns d loss / d tau
  // (r2_in: the column sums of v when the caller already has them)
  __device__ __forceinline__ static float shrink_back(const Lane& L, float* nb, float* fb, float* fb2,
                                                      const WT& v, WT& g, float tau,
                                                      const float2* r2_in = nullptr) {
    const float2 r2 = r2_in ? *r2_in : S::colsum(L, nb, v);
    __syncwarp();  // every lane has read its norms before nb is reused
    const float2 vg = colsum_vg(L, nb, v, g);
    float dtau = 0.f, c1[2], c2[2];
    const float rr[2] = {r2.x, r2.y}, vv[2] = {vg.x, vg.y};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const bool act = rr[h] > tau * tau && rr[h] > 0.f;
      const float ir = act ? rsqrtf(rr[h]) : 0.f;
      c1[h] = act ? 1.f - tau * ir : 0.f;
      c2[h] = act ? tau * ir * ir * ir * vv[h] : 0.f;
      dtau -= act ? vv[h] * ir : 0.f;
    }
    put_factors(L, fb, c1[0], c1[1]);
    put_factors(L, fb2, c2[0], c2[1]);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 a = get_factors(L, fb, j), b = get_factors(L, fb2, j);
      const float fa[4] = {a.x, a.y, a.z, a.w}, fbb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int s = 2 * j + u, f = 2 * u + h;
          g[s][h] = fmaf(fa[f], g[s][h], fbb[f] * v[s][h]);
          g[s][2 + h] = fmaf(fa[f], g[s][2 + h], fbb[f] * v[s][2 + h]);
        }
    }
    __syncwarp();
#pragma unroll
    for (int msk = 1; msk < 32; msk <<= 1) dtau += __shfl_xor_sync(0xffffffffu, dtau, msk);
    return dtau;
  }

  // w -= E X with raw (unsplit) X fragments xr[nt][lane] = (Re, Re, Im, Im)
  __device__ __forceinline__ static void update_raw(const Lane& L, const float4* xr, const float (&e)[4],
                                                    WT& w) {
    uint32_t c0h, c0l, c1h, c1l, c2h, c2l, c3h, c3l;
    split_tf32(e[0], c0h, c0l);
    split_tf32(e[1], c1h, c1l);
    split_tf32(e[2], c2h, c2l);
    split_tf32(e[3], c3h, c3l);
    const uint32_t n0h = neg_bits(c0h), n1h = neg_bits(c1h), n2h = neg_bits(c2h), n3h = neg_bits(c3h);
    const uint32_t n0l = neg_bits(c0l), n1l = neg_bits(c1l), n2l = neg_bits(c2l), n3l = neg_bits(c3l);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float4 x = xr[nt * 32 + L.lane];
      uint32_t r0h, r0l, r1h, r1l, i0h, i0l, i1h, i1l;
      split_tf32(x.x, r0h, r0l);
      split_tf32(x.y, r1h, r1l);
      split_tf32(x.z, i0h, i0l);
      split_tf32(x.w, i1h, i1l);
      mma_tf32(w[nt], n0h, n2h, n1h, n3h, r0l, r1l);
      mma_tf32(w[nt], c2h, n0h, c3h, n1h, i0l, i1l);
      mma_tf32(w[nt], n0l, n2l, n1l, n3l, r0h, r1h);
      mma_tf32(w[nt], c2l, n0l, c3l, n1l, i0h, i1h);
      mma_tf32(w[nt], n0h, n2h, n1h, n3h, r0h, r1h);
      mma_tf32(w[nt], c2h, n0h, c3h, n1h, i0h, i1h);
    }
  }

  // one forward layer l: W_l -> W_{l+1}
  __device__ __forceinline__ static void fwd_layer(const Lane& L, const Ctx& c, const TrainArgs& A,
                                                   const float4* hhi, const float4* hlo,
                                                   const float4* xf, float* nb, float* fb, int l,
                                                   float invL, WT& w) {
    float e[4];
    if constexpr (MODE == kModeProj) {
      S::shrink(L, fb, S::colsum(L, nb, w), fmaxf(__ldg(A.s.step + l), 0.f), w);
      S::template residual<true>(L, nullptr, hhi, hlo, w, c.tks, true, e);
      S::update(L, xf, e, w);
    } else {
      const float eta = __ldg(A.s.step + l) * invL;
      S::template residual<true>(L, nullptr, hhi, hlo, w, c.tks, true, e);
#pragma unroll
      for (int k = 0; k < 4; ++k) e[k] *= eta;
      S::update(L, xf, e, w);
      S::shrink(L, fb, S::colsum(L, nb, w), fmaxf(fmaxf(__ldg(A.s.lam + l), 0.f) * eta, 0.f), w);
    }
  }

  __device__ static void run(const TrainArgs& A) {
    extern __shared__ __align__(16) unsigned char smem[];
    Ctx c;
    Lane L;
    const int tid = threadIdx.x;
    c.gid = tid >> 5;
    c.g = tid & 31;
    c.b = c.g % 8;
    c.a = c.g / 8;
    c.lane = tid & 31;
    c.wig = 0;
    c.wmask = 0xffffffffu;
    c.K = KB;
    c.M = MB;
    L.lane = c.lane;
    L.g = c.lane >> 2;
    L.q = c.lane & 3;
    unsigned char* gs = smem + c.gid * GROUP_STRIDE;
    c.Hs = reinterpret_cast<float2*>(gs);
    c.Qs = reinterpret_cast<float2*>(gs + S::OFF_Q);
    c.red = reinterpret_cast<float*>(gs + S::OFF_RED);
    c.Es = reinterpret_cast<float2*>(gs + S::OFF_E);
    c.nrm = nullptr;
    c.tks = reinterpret_cast<float*>(gs + S::OFF_SC);
    c.dsc = c.tks + KB;
    c.piv = c.dsc + KB;
    c.misc = reinterpret_cast<int*>(c.piv + KB);
    c.wsum = reinterpret_cast<float*>(c.misc + 8);
    c.bar = reinterpret_cast<uint64_t*>(gs + S::OFF_BAR);
    float4* const xf = reinterpret_cast<float4*>(gs + S::OFF_XF);
    float4* const hlo = reinterpret_cast<float4*>(gs + S::OFF_LO);
    float* const nb = reinterpret_cast<float*>(gs + S::OFF_NB);
    float* const fb = reinterpret_cast<float*>(gs + S::OFF_FB);
    float* const fb2 = reinterpret_cast<float*>(gs + OFF_FB2);
    float4* const xr = MODE == kModeProj ? reinterpret_cast<float4*>(gs + OFF_XR) : nullptr;
    const float4* const hhi = reinterpret_cast<const float4*>(c.Hs);
    if (c.g == 0) mbar_init(c.bar, 1);
    fence_mbar_init();
    __syncthreads();

    const int T = A.s.T;
    const int PW = 1 + 2 * T;
    uint32_t phase = 0;
    const int64_t n_inst = A.s.B;
    const int64_t stride = (int64_t)gridDim.x * NW;
    auto issue_copy = [&](int64_t it) {
      if (c.g != 0 || it >= n_inst || (A.s.opts & OPT_STALL_COPY)) return;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(c.bar, KB * MB * 8);
      bulk_g2s(c.Hs, A.s.H + it * (int64_t)(KB * MB), KB * MB * 8, c.bar);
    };
    const int64_t first = (int64_t)blockIdx.x * NW + c.gid;
    issue_copy(first);
    WT w, g;
#pragma unroll 1
    for (int64_t inst = first; inst < n_inst; inst += stride) {
      float* const part = A.part + inst * PW;
      __syncwarp();
      if (c.g < KB) c.tks[c.g] = A.s.t[inst * A.s.t_stride + c.g];
      if (c.g == 0) c.misc[0] = mbar_wait_bounded(c.bar, phase, copy_wait_ns(A.s)) ? 1 : 0;
      __syncwarp();
      if (c.misc[0] == 0) {
        if (c.g == 0) {
          atomicAdd(A.s.err, 1ull);
          if (A.s.flags) A.s.flags[inst] = PRECODE_F_TIMEOUT;
          c.misc[1] = mbar_wait_bounded(c.bar, phase, copy_wait_ns(A.s)) ? 1 : 0;
        }
        __syncwarp();
        if (c.misc[1] == 0) return;
        for (int j = c.g; j < PW; j += 32) part[j] = 0.f;
        phase ^= 1u;
        issue_copy(inst + stride);
        continue;
      }
      if (c.g != 0) mbar_wait_bounded(c.bar, phase, copy_wait_ns(A.s));
      phase ^= 1u;

      float invL;
      const int fl = S::setup(c, L, A.s, xf, hlo, w, invL, xr);
      __syncwarp();
      if (fl & PRECODE_F_SINGULAR) {  // W_T = 0: ||S||_F^2, or ||W_gt||_F^2 with labels
        float s2 = 0.f;
        if (A.wgt) {
          s2 = sup_loss_zero(L, A.wgt + inst * (int64_t)(KB * MB));
        } else {
          for (int k = 0; k < KB; ++k) s2 += c.tks[k] * c.tks[k];
        }
        for (int j = c.g; j < PW; j += 32) part[j] = (j == 0) ? s2 : 0.f;
        if (c.g == 0 && A.s.flags) A.s.flags[inst] = fl;
        __syncwarp();
        issue_copy(inst + stride);
        continue;
      }
      float4* const cp = reinterpret_cast<float4*>(A.cp + inst * (int64_t)A.ncp * (KB * MB));
      auto store_cp = [&](int k) {
#pragma unroll
        for (int s = 0; s < 8; ++s)
          cp[(k * 8 + s) * 32 + L.lane] = make_float4(w[s][0], w[s][1], w[s][2], w[s][3]);
      };
      auto load_cp = [&](int k) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const float4 v = cp[(k * 8 + s) * 32 + L.lane];
          w[s][0] = v.x;
          w[s][1] = v.y;
          w[s][2] = v.z;
          w[s][3] = v.w;
        }
      };

      // ---- forward with checkpoints
#pragma unroll 1
      for (int l = 0; l < T; ++l) {
        if (l % A.cp_every == 0) store_cp(l / A.cp_every);
        fwd_layer(L, c, A, hhi, hlo, xf, nb, fb, l, invL, w);
      }

      // ---- loss and its gradient at W_T
      float o, rs, e[4];
      if (A.wgt) {  // supervised: ||W_T - W_gt||_F^2, g = 2 (W_T - W_gt)
        const float ls = sup_loss_grad(L, A.wgt + inst * (int64_t)(KB * MB), 1.f, w, g);
        if (c.g == 0) part[0] = ls;
      } else {
        const float2 r2 = S::colsum(L, nb, w);
        o = sqrtf(r2.x) + sqrtf(r2.y);
#pragma unroll
        for (int msk = 1; msk < 32; msk <<= 1) o += __shfl_xor_sync(0xffffffffu, o, msk);
        put_factors(L, fb, r2.x > 0.f ? A.a * rsqrtf(r2.x) : 0.f, r2.y > 0.f ? A.a * rsqrtf(r2.y) : 0.f);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 f = get_factors(L, fb, j);
          const float ff[4] = {f.x, f.y, f.z, f.w};
#pragma unroll
          for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              g[2 * j + u][h] = ff[2 * u + h] * w[2 * j + u][h];
              g[2 * j + u][2 + h] = ff[2 * u + h] * w[2 * j + u][2 + h];
            }
        }
        __syncwarp();
        S::template residual<true>(L, nullptr, hhi, hlo, w, c.tks, true, e);  // E_T
        rs = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + e[3] * e[3];
#pragma unroll
        for (int msk = 1; msk < 32; msk <<= 1) rs += __shfl_xor_sync(0xffffffffu, rs, msk);
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] *= -2.f;
        if constexpr (MODE == kModeProj)
          update_raw(L, xr, e, g);  // g += 2 E_T H^*
        else
          S::update(L, xf, e, g);
        if (c.g == 0) part[0] = A.a * o + rs;
      }

      // ---- reverse: layer l = T-1 .. 0, recomputing its input from a checkpoint
#pragma unroll 1
      for (int l = T - 1; l >= 0; --l) {
        const int k = l / A.cp_every;
        load_cp(k);
#pragma unroll 1
        for (int s = k * A.cp_every; s < l; ++s) fwd_layer(L, c, A, hhi, hlo, xf, nb, fb, s, invL, w);
        // w = W_l, the input of layer l
        if constexpr (MODE == kModeProj) {
          float eg[4];
          S::template residual<true>(L, nullptr, hhi, hlo, g, c.tks, false, eg);  // g H^T
          S::update(L, xf, eg, g);                                                // g - (g H^T) Q
          const float mu_raw = __ldg(A.s.step + l);
          const float dmu = shrink_back(L, nb, fb, fb2, w, g, fmaxf(mu_raw, 0.f));
          if (c.g == 0) part[1 + l] = mu_raw > 0.f ? dmu : 0.f;
        } else {
          const float eta = __ldg(A.s.step + l) * invL;
          const float lam_raw = __ldg(A.s.lam + l);
          const float lam = fmaxf(lam_raw, 0.f);
          const float tau = fmaxf(lam * eta, 0.f);
          float el[4], ee[4], eg[4];
          S::template residual<true>(L, nullptr, hhi, hlo, w, c.tks, true, el);  // E_l
#pragma unroll
          for (int q = 0; q < 4; ++q) ee[q] = eta * el[q];
          S::update(L, xf, ee, w);  // w = V_l
          const float dtau = shrink_back(L, nb, fb, fb2, w, g, tau);  // g = d loss / d V_l
          S::template residual<true>(L, nullptr, hhi, hlo, g, c.tks, false, eg);  // g_V H^T
          float dot = eg[0] * el[0] + eg[1] * el[1] + eg[2] * el[2] + eg[3] * el[3];
#pragma unroll
          for (int msk = 1; msk < 32; msk <<= 1) dot += __shfl_xor_sync(0xffffffffu, dot, msk);
#pragma unroll
          for (int q = 0; q < 4; ++q) eg[q] *= eta;
          S::update(L, xf, eg, g);  // g_V - eta (g_V H^T) H^*
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
        for (int j = 1 + T + c.g; j < PW; j += 32) part[j] = 0.f;
      __syncwarp();  // the channel buffer is free
      issue_copy(inst + stride);
    }
  }
};

template <int MODE, int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) train_tc_kernel(TrainArgs A) {
  TrainTC<MODE, NW>::run(A);
}

}  // namespace precode
