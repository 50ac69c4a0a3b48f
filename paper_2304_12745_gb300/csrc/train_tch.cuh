// Forward + adjoint of T projected layers with the layers' contractions as
// split-FP16 warp MMAs, K = 8 users, M = 64 antennas, one warp per instance (the
// layout, scaled units and building blocks of the split-FP16 solve kernel).
//
// The forward runs in the solve kernel's units (H' = D H, W' = b W, mu' = b mu),
// whose layer maps have the same Jacobians as the original ones, so the adjoint
// runs in them too: with g' = s dL/dW (s a power of two putting max |g'| in
// [8, 16) at W_T), every reverse step is the original one on scaled operands:
//   projection  g' <- g' - (g' H'^T) Q'      (H'^T Q' = H^T Q)
//   shrink      g' <- (1 - tau'/r') g' + (tau'/r'^3) Re(v'^H g') v'  (scale-free)
//               d tau' = -sum_active Re(v'^H g') / r'  =  s dL/dmu
// The loss and its gradient at W_T are formed in original units in FP32 (the
// gradient's 2 E_T H^* with split-TF32 MMAs on the unscaled conj(H); with labels,
// the supervised 2 (W_T - W_gt)).  W_l is
// kept (scaled) at every c-th layer and the reverse pass recomputes the layers in
// between.  Up to CP_ONCHIP checkpoints stay in tensor memory: a warp's W
// fragments are 32 registers a lane, one 32x32b store of 32 columns into the
// warp's lane quarter (warp w: quarter w % 4, column group w / 4 of 32 CP_ONCHIP
// columns); more go to a global workspace.  The host takes the shortest interval c
// whose ceil(T / c) checkpoints fit on chip when that is below ceil(sqrt(T)): at
// T = 10, c = 2 and 5 recomputed layers instead of 13.  A kernel that allocates tensor memory
// is resident once per SM, so the build runs one block of 12 warps per SM (the
// warps of three 4-warp blocks).
#pragma once

#include "solve_tch.cuh"
#include "tcgen05.cuh"
#include "train_tc.cuh"

namespace precode {

template <int NW>
struct TrainTCH {
  using SH = SolveTCH<NW>;
  using S = typename SH::S;
  using TT = TrainTC<kModeProj, NW>;
  using Ctx = typename SH::Ctx;
  using Lane = typename SH::Lane;
  using WT = typename SH::WT;
  static constexpr int KB = 8, MB = 64;
  // per warp: the split-FP16 solve kernel's layout, a second shrink-factor buffer
  // and the unscaled conj(H) B fragments for the loss gradient's E_T H^*
  static constexpr int OFF_FB2 = SH::GROUP_STRIDE;
  static constexpr int OFF_XR = OFF_FB2 + 256;
  static constexpr int GROUP_STRIDE = OFF_XR + 8 * 32 * 16;
  static constexpr int OFF_TSLOT = NW * GROUP_STRIDE;  // the block's TMEM address
  static constexpr int SMEM_BYTES = OFF_TSLOT + 16;
  static constexpr int CP_ONCHIP = 5;
  static constexpr uint32_t CP_GROUP = 32 * CP_ONCHIP;  // columns of one warp's checkpoints
  // allocation: the next power of two (at least 32) above the column groups in use
  static constexpr uint32_t pow2_at_least(uint32_t n) { return n <= 32 ? 32u : 2u * pow2_at_least((n + 1) / 2); }
  static constexpr uint32_t CP_COLS = pow2_at_least(CP_GROUP * (uint32_t)((NW + 3) / 4));
  static_assert(CP_COLS <= 512, "the checkpoints fit tensor memory");
  static_assert(NW <= 16 && (NW <= 4 || NW % 4 == 0), "warps share lane quarters by column group");
  static_assert(GROUP_STRIDE % 16 == 0, "alignment");

  // one forward layer l in scaled units: W'_l -> W'_{l+1}
  // (r2: the column sums of the input W'_l, for a reverse step that needs them)
  __device__ __forceinline__ static void fwd_layer(const Lane& L, const Ctx& c, const TrainArgs& A,
                                                   const uint4* hh, const uint4* hl, const uint4* xf,
                                                   float* nb, float* fb, int l, float beta, WT& w,
                                                   float2& r2) {
    float e[4];
    r2 = S::colsum(L, nb, w);
    S::shrink(L, fb, r2, fmaxf(__ldg(A.s.step + l), 0.f) * beta, w);
    SH::residual_h(L, hh, hl, w, e);
    if (2 * L.q == L.g) e[0] -= c.tks[L.g];
    if (2 * L.q + 1 == L.g) e[1] -= c.tks[L.g];
    SH::update_h(L, xf, e, w);
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
    c.Qs = reinterpret_cast<float2*>(gs + SH::OFF_Q);
    c.red = reinterpret_cast<float*>(gs + SH::OFF_RED);
    c.Es = reinterpret_cast<float2*>(gs + SH::OFF_E);
    c.nrm = nullptr;
    c.tks = reinterpret_cast<float*>(gs + SH::OFF_SC);
    c.dsc = c.tks + KB;
    c.piv = c.dsc + KB;
    c.misc = reinterpret_cast<int*>(c.piv + KB);
    c.wsum = reinterpret_cast<float*>(c.misc + 8);
    c.bar = reinterpret_cast<uint64_t*>(gs + SH::OFF_BAR);
    uint4* const xf = reinterpret_cast<uint4*>(gs + SH::OFF_XF);
    const uint4* const hh = reinterpret_cast<const uint4*>(gs + SH::OFF_HH);
    const uint4* const hl = reinterpret_cast<const uint4*>(gs + SH::OFF_HL);
    float* const nb = reinterpret_cast<float*>(gs + SH::OFF_NB);
    float* const fb = reinterpret_cast<float*>(gs + SH::OFF_FB);
    float* const fb2 = reinterpret_cast<float*>(gs + OFF_FB2);
    float4* const xr = reinterpret_cast<float4*>(gs + OFF_XR);
    if (c.g == 0) mbar_init(c.bar, 1);
    fence_mbar_init();
    const bool onchip = A.cp == nullptr;  // checkpoints in tensor memory
    uint32_t* const tslot = reinterpret_cast<uint32_t*>(smem + OFF_TSLOT);
    if (onchip && c.gid == 0) tc5::alloc(smem_addr(tslot), CP_COLS);
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tbase = onchip ? *tslot : 0u;
    // this warp's lane quarter and column group
    const uint32_t tcp = tbase + ((uint32_t)(32 * (c.gid & 3)) << 16) + CP_GROUP * (uint32_t)(c.gid >> 2);

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
        if (c.misc[1] == 0) break;  // the copy never landed: stop (TMEM is freed below)
        for (int j = c.g; j < PW; j += 32) part[j] = 0.f;
        phase ^= 1u;
        issue_copy(inst + stride);
        continue;
      }
      if (c.g != 0) mbar_wait_bounded(c.bar, phase, copy_wait_ns(A.s));
      phase ^= 1u;

      float beta;
      const int fl = SH::setup(c, L, A.s, xf, w, beta, xr);
      __syncwarp();
      if (fl & PRECODE_F_SINGULAR) {  // t' = b d t: back to ||t||^2 (||W_gt||^2 with labels)
        float s2 = 0.f;
        if (A.wgt) {
          s2 = TT::sup_loss_zero(L, A.wgt + inst * (int64_t)(KB * MB));
        } else {
          for (int k = 0; k < KB; ++k) s2 += (c.tks[k] * c.dsc[k]) * (c.tks[k] * c.dsc[k]);
          s2 /= beta * beta;
        }
        for (int j = c.g; j < PW; j += 32) part[j] = (j == 0) ? s2 : 0.f;
        if (c.g == 0 && A.s.flags) A.s.flags[inst] = fl;
        __syncwarp();
        issue_copy(inst + stride);
        continue;
      }
      float4* const cp = onchip ? nullptr
                                : reinterpret_cast<float4*>(A.cp + inst * (int64_t)A.ncp * (KB * MB));
      auto store_cp = [&](int k) {
        if (onchip) {
          float v[32];
#pragma unroll
          for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int i = 0; i < 4; ++i) v[4 * s + i] = w[s][i];
          tc5::st32x32b_x32(tcp + 32 * k, v);
          tc5::wait_st();
          return;
        }
#pragma unroll
        for (int s = 0; s < 8; ++s)
          cp[(k * 8 + s) * 32 + L.lane] = make_float4(w[s][0], w[s][1], w[s][2], w[s][3]);
      };
      auto load_cp = [&](int k) {
        if (onchip) {
          float v[32];
          tc5::ld32x32b_x32(tcp + 32 * k, v);
          tc5::wait_ld();
#pragma unroll
          for (int s = 0; s < 8; ++s)
#pragma unroll
            for (int i = 0; i < 4; ++i) w[s][i] = v[4 * s + i];
          return;
        }
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          const float4 v = cp[(k * 8 + s) * 32 + L.lane];
          w[s][0] = v.x;
          w[s][1] = v.y;
          w[s][2] = v.z;
          w[s][3] = v.w;
        }
      };

      // ---- forward with checkpoints (scaled units)
#pragma unroll 1
      for (int l = 0; l < T; ++l) {
        if (l % A.cp_every == 0) store_cp(l / A.cp_every);
        float2 r2;
        fwd_layer(L, c, A, hh, hl, xf, nb, fb, l, beta, w, r2);
      }

      // ---- loss and its gradient at W_T, in original units
      const float ib = 1.f / beta;
      float o, rs, e[4];
      if (A.wgt) {  // supervised: ||W_T - W_gt||_F^2, g = 2 (W_T - W_gt), W_T = w / b
        const float ls = TT::sup_loss_grad(L, A.wgt + inst * (int64_t)(KB * MB), ib, w, g);
        if (c.g == 0) part[0] = ls;
      } else {
        const float2 r2 = S::colsum(L, nb, w);
        o = sqrtf(r2.x) + sqrtf(r2.y);
#pragma unroll
        for (int msk = 1; msk < 32; msk <<= 1) o += __shfl_xor_sync(0xffffffffu, o, msk);
        o *= ib;
        // a w_m / ||w_m|| is the same in both units
        TT::put_factors(L, fb, r2.x > 0.f ? A.a * rsqrtf(r2.x) : 0.f,
                        r2.y > 0.f ? A.a * rsqrtf(r2.y) : 0.f);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float4 f = TT::get_factors(L, fb, j);
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
        SH::residual_h(L, hh, hl, w, e);  // E'_T = b E_T D
        if (2 * L.q == L.g) e[0] -= c.tks[L.g];
        if (2 * L.q + 1 == L.g) e[1] -= c.tks[L.g];
        const float d0 = c.dsc[2 * L.q] * ib, d1 = c.dsc[2 * L.q + 1] * ib;
        e[0] *= d0;
        e[2] *= d0;
        e[1] *= d1;
        e[3] *= d1;  // E_T
        rs = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + e[3] * e[3];
#pragma unroll
        for (int msk = 1; msk < 32; msk <<= 1) rs += __shfl_xor_sync(0xffffffffu, rs, msk);
#pragma unroll
        for (int k = 0; k < 4; ++k) e[k] *= -2.f;
        TT::update_raw(L, xr, e, g);  // g += 2 E_T H^*
        if (c.g == 0) part[0] = A.a * o + rs;
      }
      // g' = s g with max |g'| in [8, 16)
      float gm = 0.f;
#pragma unroll
      for (int s = 0; s < 8; ++s)
#pragma unroll
        for (int k = 0; k < 4; ++k) gm = fmaxf(gm, fabsf(g[s][k]));
      gm = SH::warp_max(gm);
      const float gs_ = 16.f * SH::inv_pow2_of(gm), igs = 1.f / gs_;
#pragma unroll
      for (int s = 0; s < 8; ++s)
#pragma unroll
        for (int k = 0; k < 4; ++k) g[s][k] *= gs_;

      // ---- reverse: layer l = T-1 .. 0, recomputing its input from a checkpoint.  The
      // last recomputed layer's input column sums (of W'_{l-1}) serve the next step,
      // whose input that is (bitwise the same values, reloaded)
      float2 r2c = make_float2(0.f, 0.f);
      int r2l = -1;
#pragma unroll 1
      for (int l = T - 1; l >= 0; --l) {
        const int k = l / A.cp_every;
        load_cp(k);
#pragma unroll 1
        for (int s = k * A.cp_every; s < l; ++s) {
          fwd_layer(L, c, A, hh, hl, xf, nb, fb, s, beta, w, r2c);
          r2l = s;
        }
        // w = W'_l, the input of layer l
        float eg[4];
        SH::residual_h(L, hh, hl, g, eg);  // g' H'^T
        SH::update_h(L, xf, eg, g);        // g' - (g' H'^T) Q'
        const float mu_raw = __ldg(A.s.step + l);
        const float dmu = TT::shrink_back(L, nb, fb, fb2, w, g, fmaxf(mu_raw, 0.f) * beta,
                                          r2l == l ? &r2c : nullptr);
        if (c.g == 0) part[1 + l] = mu_raw > 0.f ? dmu * igs : 0.f;
      }
      if (c.g == 0 && A.s.flags) A.s.flags[inst] = fl;
      for (int j = 1 + T + c.g; j < PW; j += 32) part[j] = 0.f;
      __syncwarp();  // the channel buffer is free
      issue_copy(inst + stride);
    }
    tc5::fence_before_sync();
    __syncthreads();
    if (onchip && c.gid == 0) tc5::dealloc(tbase, CP_COLS);
  }
};

template <int NW, int MINB>
__global__ void __launch_bounds__(NW * 32, MINB) train_tch_kernel(TrainArgs A) {
  TrainTCH<NW>::run(A);
}

}  // namespace precode
