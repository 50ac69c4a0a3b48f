// Tensor-core variant of the persistent solve kernel for K = 8 users, M = 64
// antennas: one warp per instance, both contractions of a layer as warp-level
// MMAs (m16n8k8, TF32 inputs, FP32 accumulation) with a three-term TF32 split
// (x = hi + lo; a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi), which keeps products
// accurate to about 2^-21 relative, close to FP32.
//
// Real forms (Re/Im stacked):
//   E = W H^T:   [E_re; E_im] (16x8)  = [[Wr, -Wi], [Wi, Wr]] (16x128) . [Hr^T; Hi^T] (128x8)
//   W -= E X:    [W_re; W_im] (16x64) += -[[E_re, -E_im], [E_im, E_re]] (16x16) . [X_re; X_im] (16x64)
// with X = Q = G^{-T} H^* (projected layer) or eta conj(H) (paper layer).
// Lane (g, q) = (lane / 4, lane % 4) holds user g's W at antennas 8s + 2q + h
// (s = 0..7, h = 0, 1).  Ordering the MMA reduction dimension within each block
// of 8 as 2q (columns q) and 2q + 1 (columns q + 4) makes:
//   * the A fragments of the first MMA exactly the lane's own W entries, and its
//     B fragments the lane's own H entries (user g's row of H);
//   * the accumulator fragments of the first MMA (E[g][2q], E[g][2q+1]) exactly
//     the A fragments of the second;
//   * the accumulator fragments of the second MMA exactly the lane's W entries.
// So no data moves between lanes for the contractions; only the per-antenna
// column norms of the shrink reduce over the 8 lanes of a column (shuffles).
#pragma once

#include "solve.cuh"

namespace precode {

// x = hi + lo exactly: hi keeps the 10 explicit mantissa bits a TF32 operand
// carries (low 13 bits cleared), lo = x - hi is exact in FP32; the MMA reads
// lo's top TF32 bits, so a b is resolved to about 2^-21 relative.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = __float_as_uint(x) & 0xffffe000u;
  lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ uint32_t neg_bits(uint32_t x) { return x ^ 0x80000000u; }

// d += a . b  (m16n8k8, row.col, TF32 in, FP32 accumulate)
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

template <int MODE, int NW, bool DB>
struct SolveTC : SolveKernel<MODE, 8, 64, 4, 8, 8, true, NW, true, DB> {
  using Base = SolveKernel<MODE, 8, 64, 4, 8, 8, true, NW, true, DB>;
  using C = typename Base::C;
  using Ctx = typename Base::Ctx;
  static constexpr int KB = 8, MB = 64;
  // Per-lane pre-split B fragments of the second contraction, [nt][hi/lo][lane]
  // float4 (8 KB).  They live in the Q + reduction buffers, which only the setup uses.
  static constexpr int XF_BYTES = 8 * 2 * 32 * 16;
  static_assert(C::Q_BYTES + C::RED_BYTES >= XF_BYTES || MODE == kModePGD, "fragment area");
  static constexpr int XF_OFF = MODE == kModeProj ? C::Q_OFF : C::GROUP_BYTES;
  static constexpr int GROUP_STRIDE =
      MODE == kModeProj ? C::GROUP_BYTES : align_up(C::GROUP_BYTES + XF_BYTES, 16);
  static constexpr int SMEM_BYTES = C::GROUPS * GROUP_STRIDE;

  struct Lane {
    int g, q, lane;
  };
  // W in MMA accumulator order: w[s] = (Re W[g][8s+2q], Re W[g][8s+2q+1],
  //                                     Im W[g][8s+2q], Im W[g][8s+2q+1])
  using WT = float[8][4];

  __device__ __forceinline__ static void colnorm2(const WT& w, float (&r2)[8][2]) {
#pragma unroll
    for (int s = 0; s < 8; ++s)
#pragma unroll
      for (int h = 0; h < 2; ++h) r2[s][h] = fmaf(w[s][h], w[s][h], w[s][2 + h] * w[s][2 + h]);
#pragma unroll
    for (int msk = 4; msk < 32; msk <<= 1)
#pragma unroll
      for (int s = 0; s < 8; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h) r2[s][h] += __shfl_xor_sync(0xffffffffu, r2[s][h], msk);
  }

  __device__ __forceinline__ static void shrink(WT& w, const float (&r2)[8][2], float tau) {
    const float tau2 = tau * tau;
#pragma unroll
    for (int s = 0; s < 8; ++s)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float f = (r2[s][h] > tau2) ? (1.f - tau * rsqrtf(r2[s][h])) : 0.f;
        w[s][h] *= f;
        w[s][2 + h] *= f;
      }
  }

  // E = W H^T (minus S on the diagonal when sub_s): returns the lane's fragment
  // e = (E_re[g][2q], E_re[g][2q+1], E_im[g][2q], E_im[g][2q+1]).  Four blocks of
  // 8 antennas at a time, their MMAs issued term by term over four accumulators.
  __device__ __forceinline__ static void residual(const Lane& L, const float2* Hs, const WT& w,
                                                  const float* tks, bool sub_s, float (&e)[4]) {
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[i][k] = 0.f;
#pragma unroll
    for (int s0 = 0; s0 < 8; s0 += 4) {
      uint32_t bh[4][4], bl[4][4], ah[4][4], al[4][4];  // [block][hr0 hr1 hi0 hi1 / r0 i0 r1 i1]
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int s = s0 + u;
        const float4 hv = *reinterpret_cast<const float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
        split_tf32(hv.x, bh[u][0], bl[u][0]);
        split_tf32(hv.z, bh[u][1], bl[u][1]);
        split_tf32(hv.y, bh[u][2], bl[u][2]);
        split_tf32(hv.w, bh[u][3], bl[u][3]);
        split_tf32(w[s][0], ah[u][0], al[u][0]);  // Re W, h = 0
        split_tf32(w[s][2], ah[u][1], al[u][1]);  // Im W, h = 0
        split_tf32(w[s][1], ah[u][2], al[u][2]);  // Re W, h = 1
        split_tf32(w[s][3], ah[u][3], al[u][3]);  // Im W, h = 1
      }
      // real block (kb = s): A = (re0, im0, re1, im1), B = (hr0, hr1)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(acc[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bl[u][0], bl[u][1]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(acc[u], al[u][0], al[u][1], al[u][2], al[u][3], bh[u][0], bh[u][1]);
      // imaginary block (kb = s + 8): A = (-im0, re0, -im1, re1), B = (hi0, hi1)
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(acc[u], neg_bits(ah[u][1]), ah[u][0], neg_bits(ah[u][3]), ah[u][2], bl[u][2],
                 bl[u][3]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(acc[u], neg_bits(al[u][1]), al[u][0], neg_bits(al[u][3]), al[u][2], bh[u][2],
                 bh[u][3]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(acc[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bh[u][0], bh[u][1]);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(acc[u], neg_bits(ah[u][1]), ah[u][0], neg_bits(ah[u][3]), ah[u][2], bh[u][2],
                 bh[u][3]);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) e[k] = (acc[0][k] + acc[1][k]) + (acc[2][k] + acc[3][k]);
    if (sub_s) {
      if (2 * L.q == L.g) e[0] -= tks[L.g];
      if (2 * L.q + 1 == L.g) e[1] -= tks[L.g];
    }
  }

  // W -= E X with the lane's E fragment e and the pre-split X fragments; four
  // antenna tiles at a time, term by term.
  __device__ __forceinline__ static void update(const Lane& L, const float4* xf, const float (&e)[4],
                                                WT& w) {
    uint32_t c0h, c0l, c1h, c1l, c2h, c2l, c3h, c3l;
    split_tf32(e[0], c0h, c0l);
    split_tf32(e[1], c1h, c1l);
    split_tf32(e[2], c2h, c2l);
    split_tf32(e[3], c3h, c3l);
    // -A2: k-step 0 = (-c0, -c2, -c1, -c3), k-step 1 = (c2, -c0, c3, -c1)
    const uint32_t n0h = neg_bits(c0h), n1h = neg_bits(c1h), n2h = neg_bits(c2h),
                   n3h = neg_bits(c3h);
    const uint32_t n0l = neg_bits(c0l), n1l = neg_bits(c1l), n2l = neg_bits(c2l),
                   n3l = neg_bits(c3l);
#pragma unroll
    for (int nt0 = 0; nt0 < 8; nt0 += 4) {
      float4 xh[4], xl[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        xh[u] = xf[((nt0 + u) * 2 + 0) * 32 + L.lane];
        xl[u] = xf[((nt0 + u) * 2 + 1) * 32 + L.lane];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(w[nt0 + u], n0h, n2h, n1h, n3h, __float_as_uint(xl[u].x), __float_as_uint(xl[u].y));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(w[nt0 + u], n0l, n2l, n1l, n3l, __float_as_uint(xh[u].x), __float_as_uint(xh[u].y));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(w[nt0 + u], c2h, n0h, c3h, n1h, __float_as_uint(xl[u].z), __float_as_uint(xl[u].w));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(w[nt0 + u], c2l, n0l, c3l, n1l, __float_as_uint(xh[u].z), __float_as_uint(xh[u].w));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(w[nt0 + u], n0h, n2h, n1h, n3h, __float_as_uint(xh[u].x), __float_as_uint(xh[u].y));
#pragma unroll
      for (int u = 0; u < 4; ++u)
        mma_tf32(w[nt0 + u], c2h, n0h, c3h, n1h, __float_as_uint(xh[u].z), __float_as_uint(xh[u].w));
    }
  }

  __device__ static void run(const SolveArgs& A) {
    extern __shared__ __align__(16) unsigned char smem[];
    Ctx c;
    Lane L;
    const int tid = threadIdx.x;
    c.gid = tid >> 5;
    c.g = tid & 31;
    c.b = c.g % 8;  // the base kernel's lane grid, used by the shared setup code
    c.a = c.g / 8;
    c.lane = tid & 31;
    c.wig = 0;
    c.wmask = 0xffffffffu;
    L.lane = c.lane;
    L.g = c.lane >> 2;
    L.q = c.lane & 3;
    unsigned char* gs = smem + c.gid * GROUP_STRIDE;
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
    c.Hs = reinterpret_cast<float2*>(gs + C::H_OFF);
    float4* xf = reinterpret_cast<float4*>(gs + XF_OFF);
    constexpr int NHB = C::NHB;
    if (c.g == 0)
      for (int q = 0; q < NHB; ++q) mbar_init(c.bar + q, 1);
    fence_mbar_init();
    __syncthreads();

    float2* const hbuf0 = reinterpret_cast<float2*>(gs + C::H_OFF);
    uint32_t phases = 0;
    const int64_t n_inst = A.tbl ? (int64_t)(*A.count) : A.B;
    const int64_t stride = (int64_t)gridDim.x * C::GROUPS;
    auto locate = [&](int64_t it, int64_t& inst, int64_t& h_off, int64_t& w_off, int64_t& t_off) {
      if (A.tbl) {
        inst = A.index[it];
        const InstDesc d = A.tbl[inst];
        h_off = d.h_off;
        w_off = d.w_off;
        t_off = d.t_off;
      } else {
        inst = it;
        h_off = it * (int64_t)(KB * MB);
        w_off = h_off;
        t_off = it * A.t_stride;
      }
    };
    auto issue_copy = [&](int64_t it, int qb) {
      if (c.g != 0 || it >= n_inst) return;
      int64_t inst, h_off, w_off, t_off;
      locate(it, inst, h_off, w_off, t_off);
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(c.bar + qb, KB * MB * 8);
      bulk_g2s(hbuf0 + qb * (KB * MB), A.H + h_off, KB * MB * 8, c.bar + qb);
    };
    const int64_t first = (int64_t)blockIdx.x * C::GROUPS + c.gid;
    for (int qb = 0; qb < NHB; ++qb) issue_copy(first + qb * stride, qb);
    int cur = 0;
    WT w;
    float r2[8][2], e[4];
#pragma unroll 1
    for (int64_t it = first; it < n_inst; it += stride, cur = (cur + 1) % NHB) {
      int64_t inst, h_off, w_off, t_off;
      locate(it, inst, h_off, w_off, t_off);
      c.K = KB;
      c.M = MB;
      c.Hs = hbuf0 + cur * (KB * MB);
      const uint32_t par = (phases >> cur) & 1u;
      __syncwarp();
      if (c.g < KB) c.tks[c.g] = A.t[t_off + c.g];
      if (c.g == 0) c.misc[0] = mbar_wait_bounded(c.bar + cur, par, kCopyWaitNs) ? 1 : 0;
      __syncwarp();
      if (c.misc[0] == 0) {
        if (c.g == 0) {
          atomicAdd(A.err, 1ull);
          if (A.flags) A.flags[inst] = PRECODE_F_TIMEOUT;
          c.misc[1] = mbar_wait_bounded(c.bar + cur, par, kCopyWaitNs) ? 1 : 0;
        }
        __syncwarp();
        if (c.misc[1] == 0) return;
        phases ^= 1u << cur;
        issue_copy(it + NHB * stride, cur);
        continue;
      }
      if (c.g != 0) mbar_wait_bounded(c.bar + cur, par, kCopyWaitNs);
      phases ^= 1u << cur;

      // ---- setup: lane's own conj(H) entries (user g, antennas 8s + 2q + h)
      int fl = 0;
      float invL = 1.f;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float4 hv = *reinterpret_cast<const float4*>(c.Hs + L.g * MB + 8 * s + 2 * L.q);
        w[s][0] = hv.x;
        w[s][1] = hv.z;
        w[s][2] = -hv.y;
        w[s][3] = -hv.w;
      }
      const bool need_gram = (MODE == kModeProj) || (A.opts & OPT_STEP_NORMALISED);
      if (need_gram) {
        residual(L, c.Hs, w, c.tks, false, e);  // sum_m conj(H_gm) H_jm = G^T
        *reinterpret_cast<float4*>(c.Es + L.g * KB + 2 * L.q) = make_float4(e[0], e[2], e[1], e[3]);
        __syncwarp();
        if constexpr (MODE == kModeProj) {
          typename Base::WReg wtmp;
          fl = Base::setup_proj(c, wtmp, A.cond_thr);  // Q = G^{-T} H^* into Qs (natural)
        } else {
          invL = Base::inv_gershgorin(c);
        }
      }
      const bool singular = (fl & PRECODE_F_SINGULAR) != 0;
      // fragments X[2q][8nt+g], X[2q+1][8nt+g] of the update, read before the
      // fragment area (which overlaps Q) is written
      {
        const float2* X = (MODE == kModeProj) ? c.Qs : c.Hs;
        const float csign = (MODE == kModeProj) ? 1.f : -1.f;  // paper layer: X = conj(H)
        float2 x0[8], x1[8];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          x0[nt] = singular ? make_float2(0.f, 0.f) : X[(2 * L.q) * MB + 8 * nt + L.g];
          x1[nt] = singular ? make_float2(0.f, 0.f) : X[(2 * L.q + 1) * MB + 8 * nt + L.g];
        }
        if constexpr (MODE == kModeProj) {  // W^(0) = S Q
          const float tg = c.tks[L.g];
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const float4 qv = singular ? make_float4(0.f, 0.f, 0.f, 0.f)
                                       : *reinterpret_cast<const float4*>(c.Qs + L.g * MB + 8 * s + 2 * L.q);
            w[s][0] = tg * qv.x;
            w[s][1] = tg * qv.z;
            w[s][2] = tg * qv.y;
            w[s][3] = tg * qv.w;
          }
        }
        __syncwarp();
#pragma unroll
        for (int nt = 0; nt < 8; ++nt) {
          uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
          split_tf32(x0[nt].x, h0, l0);
          split_tf32(x1[nt].x, h1, l1);
          split_tf32(csign * x0[nt].y, h2, l2);
          split_tf32(csign * x1[nt].y, h3, l3);
          xf[(nt * 2 + 0) * 32 + L.lane] = make_float4(__uint_as_float(h0), __uint_as_float(h1),
                                                       __uint_as_float(h2), __uint_as_float(h3));
          xf[(nt * 2 + 1) * 32 + L.lane] = make_float4(__uint_as_float(l0), __uint_as_float(l1),
                                                       __uint_as_float(l2), __uint_as_float(l3));
        }
      }
      __syncwarp();

      // ---- layers
      const int T = A.T;
      float rs = 0.f;
      if (!singular) {
#pragma unroll 1
        for (int l = 0; l < T; ++l) {
          if constexpr (MODE == kModeProj) {
            colnorm2(w, r2);
            shrink(w, r2, fmaxf(__ldg(A.step + l), 0.f));
            residual(L, c.Hs, w, c.tks, true, e);
            update(L, xf, e, w);
          } else {
            const float eta = __ldg(A.step + l) * invL;
            residual(L, c.Hs, w, c.tks, true, e);
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] *= eta;
            update(L, xf, e, w);
            colnorm2(w, r2);
            shrink(w, r2, fmaxf(fmaxf(__ldg(A.lam + l), 0.f) * eta, 0.f));
          }
        }
        if (A.resid) {
          residual(L, c.Hs, w, c.tks, true, e);
          rs = e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + e[3] * e[3];
#pragma unroll
          for (int msk = 1; msk < 32; msk <<= 1) rs += __shfl_xor_sync(0xffffffffu, rs, msk);
        }
      } else {
#pragma unroll
        for (int s = 0; s < 8; ++s)
#pragma unroll
          for (int k = 0; k < 4; ++k) w[s][k] = 0.f;
        for (int k = 0; k < KB; ++k) rs += c.tks[k] * c.tks[k];
      }

      // ---- channel buffer free: next copy, then objective and W
      __syncwarp();
      issue_copy(it + NHB * stride, cur);
      colnorm2(w, r2);
      float o = 0.f;
#pragma unroll
      for (int s = 0; s < 8; ++s) o += sqrtf(r2[s][0]) + sqrtf(r2[s][1]);
      o += __shfl_xor_sync(0xffffffffu, o, 1);
      o += __shfl_xor_sync(0xffffffffu, o, 2);
#pragma unroll
      for (int s = 0; s < 8; ++s)
        *reinterpret_cast<float4*>(A.W + w_off + L.g * MB + 8 * s + 2 * L.q) =
            make_float4(w[s][0], w[s][2], w[s][1], w[s][3]);
      if (c.g == 0) {
        if (!(o < FLT_MAX) || !(rs < FLT_MAX)) fl |= PRECODE_F_NONFINITE;
        if (A.obj) A.obj[inst] = o;
        if (A.resid) A.resid[inst] = sqrtf(rs);
        if (A.flags) A.flags[inst] = fl;
      }
    }
  }
};

template <int MODE, int NW, int MINB, bool DB>
__global__ void __launch_bounds__(NW * 32, MINB) solve_tc_kernel(SolveArgs A) {
  SolveTC<MODE, NW, DB>::run(A);
}

}  // namespace precode
