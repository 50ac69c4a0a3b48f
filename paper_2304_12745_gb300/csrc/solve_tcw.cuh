// Multi-warp tensor-core solve kernel for buckets of up to KB = 8 KW users and
// exactly MB antennas (MB a multiple of 64).  One CTA of KW warps works on one
// instance at a time (persistent over instances).  Instances with K < KB users
// run padded: the missing channel rows are zero, their targets zero and their
// Gram diagonal one, so their W rows stay exactly zero and the real users'
// iteration is unchanged.  Warp w owns users
// 8w .. 8w + 7 across all antennas; lane (g, q) = (lane / 4, lane % 4) holds user
// 8w + g at antennas 8s + 2q + {0, 1} (s < M / 8) in the m16n8k8 accumulator
// order (Re, Re, Im, Im), as in the K = 8 kernel, so both contractions take their
// operands lane-locally and the residual needs no sum across warps:
//   residual         E[8w+g][:] = W[8w+g][:] H^T - S        (the warp's rows)
//   projected layer  F = E G^{-T}  (K x K),   W = X - F conj(H)   (= X - E Q)
//   paper layer      F = eta E,               V = W - F conj(H)
// All products are split TF32 (a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi, FP32
// accumulation).  Shared memory holds the raw channel (rows padded by 16 bytes,
// which keeps both access patterns of the contractions nearly conflict free),
// G^{-T}, the per-warp F tiles and the column-norm partials; H's TF32 parts are
// formed on the fly.  The per-antenna norms of the shrink sum over all K users:
// each warp reduces its 8 users with a shuffle reduce-scatter and the KW
// partials meet in shared memory (one CTA barrier per layer).
// Setup of the projected layer: Gram matrix by MMA, equilibrated Gauss-Jordan
// inverse over the CTA in FP32 (pivot spread = condition estimate), FP64
// Gauss-Jordan when the estimate exceeds the threshold.
#pragma once

#include "solve.cuh"
#include "tf32mma.cuh"

namespace precode {

template <int KW, int MB_>
struct TcwCfg {
  static constexpr int KB = 8 * KW, MB = MB_, NS = MB / 8, NT = 32 * KW;
  static_assert(MB % 64 == 0, "8 antenna blocks per lane at least (the reduce-scatter halves them 3 times)");
  static constexpr int RSF = MB + 2;                      // channel row stride in float2 (+16 B)
  static constexpr int H_BYTES = KB * RSF * 8;
  static constexpr int E_BYTES = KB * KB * 8;             // Gram, then G^{-T} (float2, natural)
  static constexpr int A64_BYTES = KB * KB * 16;          // FP64 path matrix (double2)
  static constexpr int S64_BYTES = 2 * KB * 16 + KB * 8;  // FP64 pivot row / column, diagonal
  static constexpr int GF_BYTES = KW * KW * 32 * 16;      // G^{-T} B fragments [kt][ct][lane]
  static constexpr int NPR = 2 * NS + 4;                  // padded norm row (floats)
  static constexpr int NP_BYTES = 2 * KW * 4 * NPR * 4;   // norm partials [parity][warp][q]
  static constexpr int FB_BYTES = KW * 4 * NPR * 4;       // shrink factors [warp][q]
  static constexpr int FT_BYTES = KW * KW * 32 * 16;      // F tiles [warp][kt][lane]
  static constexpr int LAYER_BYTES = GF_BYTES + NP_BYTES + FB_BYTES + FT_BYTES;
  static constexpr int X_BYTES =
      LAYER_BYTES > A64_BYTES + S64_BYTES ? LAYER_BYTES : A64_BYTES + S64_BYTES;
  static constexpr int OFF_E = H_BYTES;
  static constexpr int OFF_X = OFF_E + E_BYTES;  // setup: FP64 scratch; layers: the rest
  static constexpr int OFF_GF = OFF_X;
  static constexpr int OFF_NP = OFF_GF + GF_BYTES;
  static constexpr int OFF_FB = OFF_NP + NP_BYTES;
  static constexpr int OFF_FT = OFF_FB + FB_BYTES;
  static constexpr int OFF_S64 = OFF_X + A64_BYTES;
  static constexpr int OFF_SC = OFF_X + X_BYTES;  // t[KB] dsc[KB] rowp[KB] colp[KB] misc[8] wred[KW]
  static constexpr int SC_BYTES = align_up((2 * KB + 4 * KB + 8 + KW) * 4, 16);
  static constexpr int OFF_BAR = OFF_SC + SC_BYTES;
  static constexpr int SMEM_BYTES = align_up(OFF_BAR + 8, 16);
  static_assert((RSF * 8) % 16 == 0 && OFF_E % 16 == 0 && OFF_X % 16 == 0, "16-byte alignment");
};

template <int MODE, int KW, int MB_>
struct SolveTCW {
  using C = TcwCfg<KW, MB_>;
  static constexpr int KB = C::KB, MB = C::MB, NS = C::NS, NT = C::NT, RSF = C::RSF;
  static constexpr unsigned FULL = 0xffffffffu;

  struct Lane {
    int w, g, q, lane, tid;
  };
  using WT = float[NS][4];

  // --------------------------------------------------------------- residual
  // E tile ct of the warp's rows: e = (E_re[g][8ct+2q], E_re[g][8ct+2q+1],
  // E_im[g][8ct+2q], E_im[g][8ct+2q+1]) with E = A H^T, A = W (or conj(H)'s own
  // rows for the Gram matrix), over all antenna blocks.  Every MMA takes the
  // same A quad (Re, Im rows); products with Re H go to ar, with Im H to ai, and
  //   E_re = [ar]_row g - [ai]_row g+8,   E_im = [ai]_row g + [ar]_row g+8.
  // Two accumulator pairs (even and odd blocks).
  template <bool A_FROM_H>
  __device__ __forceinline__ static void e_tile(const Lane& L, const float2* Hs, const WT& w, int ct,
                                                float (&e)[4]) {
    float ar[2][4], ai[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) ar[i][k] = ai[i][k] = 0.f;
    const float2* hb = Hs + (8 * ct + L.g) * RSF + 2 * L.q;
    const float2* ha = Hs + (8 * L.w + L.g) * RSF + 2 * L.q;
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      float a0, a1, a2, a3;  // A quad: (Re, Im) at antenna 8s + 2q, then at 8s + 2q + 1
      if constexpr (A_FROM_H) {
        const float4 v = *reinterpret_cast<const float4*>(ha + 8 * s);
        a0 = v.x;
        a1 = -v.y;
        a2 = v.z;
        a3 = -v.w;
      } else {
        a0 = w[s][0];
        a1 = w[s][2];
        a2 = w[s][1];
        a3 = w[s][3];
      }
      uint32_t ah[4], al[4], bh[4], bl[4];
      split_tf32_ordered(a0, ah[0], al[0]);
      split_tf32_ordered(a1, ah[1], al[1]);
      split_tf32_ordered(a2, ah[2], al[2]);
      split_tf32_ordered(a3, ah[3], al[3]);
      const float4 hv = *reinterpret_cast<const float4*>(hb + 8 * s);
      split_tf32_ordered(hv.x, bh[0], bl[0]);  // Re H[8ct+g][8s+2q]
      split_tf32_ordered(hv.z, bh[1], bl[1]);  // Re H[8ct+g][8s+2q+1]
      split_tf32_ordered(hv.y, bh[2], bl[2]);  // Im
      split_tf32_ordered(hv.w, bh[3], bl[3]);
      float (&r)[4] = ar[s & 1];
      float (&i)[4] = ai[s & 1];
      // A = (re0, im0, re1, im1) throughout; B = (Re, Re) into r, (Im, Im) into i
      mma_tf32(r, ah[0], ah[1], ah[2], ah[3], bl[0], bl[1]);
      mma_tf32(i, ah[0], ah[1], ah[2], ah[3], bl[2], bl[3]);
      mma_tf32(r, al[0], al[1], al[2], al[3], bh[0], bh[1]);
      mma_tf32(i, al[0], al[1], al[2], al[3], bh[2], bh[3]);
      mma_tf32(r, ah[0], ah[1], ah[2], ah[3], bh[0], bh[1]);
      mma_tf32(i, ah[0], ah[1], ah[2], ah[3], bh[2], bh[3]);
    }
    float r[4], im[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      r[k] = ar[0][k] + ar[1][k];
      im[k] = ai[0][k] + ai[1][k];
    }
    e[0] = r[0] - im[2];
    e[1] = r[1] - im[3];
    e[2] = im[0] + r[2];
    e[3] = im[1] + r[3];
  }

  // Subtract S on the diagonal (column tile ct == w, local column 2q or 2q + 1 == g).
  __device__ __forceinline__ static void sub_s(const Lane& L, const float* tks, int ct,
                                               float (&e)[4]) {
    if (ct == L.w) {
      if (2 * L.q == L.g) e[0] -= tks[8 * L.w + L.g];
      if (2 * L.q + 1 == L.g) e[1] -= tks[8 * L.w + L.g];
    }
  }

  // Subtract the full target S~^T (rows 8w + g, columns 8ct + 2q, 8ct + 2q + 1) of
  // an instance solved in the orthonormal basis (St: [KB][KB] float2, natural).
  __device__ __forceinline__ static void sub_st(const Lane& L, const float2* St, int ct,
                                                float (&e)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(St + (8 * L.w + L.g) * KB + 8 * ct + 2 * L.q);
    e[0] -= v.x;
    e[1] -= v.z;
    e[2] -= v.y;
    e[3] -= v.w;
  }

  // ----------------------------------------------------------------- update
  // W[8w+g][:] -= F X with X = conj(H): for each user tile kt the warp's F tile
  // (A operand, from shared memory, split here), then every antenna tile nt with
  // B = (X[8kt+2q][8nt+g], X[8kt+2q+1][8nt+g]) read from the raw channel.
  __device__ __forceinline__ static void update(const Lane& L, const float2* Hs, const float4* ft,
                                                WT& w) {
#pragma unroll 1
    for (int kt = 0; kt < KW; ++kt) {
      const float4 f = ft[kt * 32 + L.lane];
      uint32_t c0h, c0l, c1h, c1l, c2h, c2l, c3h, c3l;
      split_tf32_ordered(f.x, c0h, c0l);
      split_tf32_ordered(f.y, c1h, c1l);
      split_tf32_ordered(f.z, c2h, c2l);
      split_tf32_ordered(f.w, c3h, c3l);
      const uint32_t n0h = neg_bits(c0h), n1h = neg_bits(c1h), n2h = neg_bits(c2h),
                     n3h = neg_bits(c3h);
      const uint32_t n0l = neg_bits(c0l), n1l = neg_bits(c1l), n2l = neg_bits(c2l),
                     n3l = neg_bits(c3l);
      const float2* x0 = Hs + (8 * kt + 2 * L.q) * RSF + L.g;
      const float2* x1 = x0 + RSF;
#pragma unroll
      for (int nt = 0; nt < NS; ++nt) {
        const float2 h0 = x0[8 * nt], h1 = x1[8 * nt];
        uint32_t r0h, r0l, r1h, r1l, i0h, i0l, i1h, i1l;
        split_tf32_ordered(h0.x, r0h, r0l);
        split_tf32_ordered(h1.x, r1h, r1l);
        split_tf32_ordered(-h0.y, i0h, i0l);
        split_tf32_ordered(-h1.y, i1h, i1l);
        // -A: k-step 0 (X_re) = (-c0, -c2, -c1, -c3), k-step 1 (X_im) = (c2, -c0, c3, -c1)
        mma_tf32(w[nt], n0h, n2h, n1h, n3h, r0l, r1l);
        mma_tf32(w[nt], c2h, n0h, c3h, n1h, i0l, i1l);
        mma_tf32(w[nt], n0l, n2l, n1l, n3l, r0h, r1h);
        mma_tf32(w[nt], c2l, n0l, c3l, n1l, i0h, i1h);
        mma_tf32(w[nt], n0h, n2h, n1h, n3h, r0h, r1h);
        mma_tf32(w[nt], c2h, n0h, c3h, n1h, i0h, i1h);
      }
    }
  }

  // ------------------------------------------------------ residual and F
  // E tile by tile; projected layer: F = E G^{-T} accumulated as each E tile
  // completes (gf: G^{-T} B fragments (M_re[8kt+2q][8ct+g], M_re[8kt+2q+1][8ct+g],
  // M_im[..], M_im[..]) at [kt][ct][lane]); paper layer: F = eta E.  F tiles go to
  // the warp's ft.  Returns sum |E|^2 over the lane's entries.
  __device__ __forceinline__ static float residual_f(const Lane& L, const float2* Hs, const float4* gf,
                                                     const float* tks, float eta, const WT& w,
                                                     float4* ft, const float2* St = nullptr) {
    float fa[KW][4];
#pragma unroll
    for (int i = 0; i < KW; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) fa[i][k] = 0.f;
    float ss = 0.f;
#pragma unroll 1
    for (int ct = 0; ct < KW; ++ct) {
      float e[4];
      e_tile<false>(L, Hs, w, ct, e);
      if (St)
        sub_st(L, St, ct, e);
      else
        sub_s(L, tks, ct, e);
      ss += e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + e[3] * e[3];
      if constexpr (MODE == kModeProj) {
        uint32_t c0h, c0l, c1h, c1l, c2h, c2l, c3h, c3l;
        split_tf32_ordered(e[0], c0h, c0l);
        split_tf32_ordered(e[1], c1h, c1l);
        split_tf32_ordered(e[2], c2h, c2l);
        split_tf32_ordered(e[3], c3h, c3l);
        // +A: k-step re = (c0, c2, c1, c3), k-step im = (-c2, c0, -c3, c1)
#pragma unroll
        for (int cp = 0; cp < KW; ++cp) {
          const float4 m = gf[(ct * KW + cp) * 32 + L.lane];
          uint32_t m0h, m0l, m1h, m1l, m2h, m2l, m3h, m3l;
          split_tf32_ordered(m.x, m0h, m0l);
          split_tf32_ordered(m.y, m1h, m1l);
          split_tf32_ordered(m.z, m2h, m2l);
          split_tf32_ordered(m.w, m3h, m3l);
          mma_tf32(fa[cp], c0h, c2h, c1h, c3h, m0l, m1l);
          mma_tf32(fa[cp], neg_bits(c2h), c0h, neg_bits(c3h), c1h, m2l, m3l);
          mma_tf32(fa[cp], c0l, c2l, c1l, c3l, m0h, m1h);
          mma_tf32(fa[cp], neg_bits(c2l), c0l, neg_bits(c3l), c1l, m2h, m3h);
          mma_tf32(fa[cp], c0h, c2h, c1h, c3h, m0h, m1h);
          mma_tf32(fa[cp], neg_bits(c2h), c0h, neg_bits(c3h), c1h, m2h, m3h);
        }
      } else {
        ft[ct * 32 + L.lane] = make_float4(eta * e[0], eta * e[1], eta * e[2], eta * e[3]);
      }
    }
    if constexpr (MODE == kModeProj) {
#pragma unroll
      for (int cp = 0; cp < KW; ++cp)
        ft[cp * 32 + L.lane] = make_float4(fa[cp][0], fa[cp][1], fa[cp][2], fa[cp][3]);
    }
    __syncwarp();
    return ss;
  }

  // Residual only (for the reported ||H W^T - S||_F): sum |E|^2 over the lane's entries.
  __device__ __forceinline__ static float residual_ss(const Lane& L, const float2* Hs,
                                                      const float* tks, const WT& w) {
    float ss = 0.f;
#pragma unroll 1
    for (int ct = 0; ct < KW; ++ct) {
      float e[4];
      e_tile<false>(L, Hs, w, ct, e);
      sub_s(L, tks, ct, e);
      ss += e[0] * e[0] + e[1] * e[1] + e[2] * e[2] + e[3] * e[3];
    }
    return ss;
  }

  // ---------------------------------------------------------- column norms
  // One halving step of the reduce-scatter over the 8 lanes of a column: the
  // lane keeps half of its values (the half selected by its bit b) and adds the
  // partner's copy of that half.
  template <int HALF>
  __device__ __forceinline__ static void rs_step(float* v, int b, int mask) {
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
      const float send = b ? v[j] : v[j + HALF];
      const float keep = b ? v[j + HALF] : v[j];
      v[j] = keep + __shfl_xor_sync(FULL, send, mask);
    }
  }

  // NQ = NS / 4 consecutive floats per lane after the reduce-scatter: stored and
  // loaded 16, 8 or 4 bytes at a time as NQ allows.
  static constexpr int NQ = NS / 4;
  __device__ __forceinline__ static void st_nq(float* dst, const float* v) {
    if constexpr (NQ % 4 == 0) {
#pragma unroll
      for (int c = 0; c < NQ / 4; ++c)
        *reinterpret_cast<float4*>(dst + 4 * c) = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
    } else {
#pragma unroll
      for (int c = 0; c < NQ / 2; ++c)
        *reinterpret_cast<float2*>(dst + 2 * c) = make_float2(v[2 * c], v[2 * c + 1]);
    }
  }
  __device__ __forceinline__ static void add_nq(const float* src, float* r) {
    if constexpr (NQ % 4 == 0) {
#pragma unroll
      for (int c = 0; c < NQ / 4; ++c) {
        const float4 p = *reinterpret_cast<const float4*>(src + 4 * c);
        r[4 * c] += p.x;
        r[4 * c + 1] += p.y;
        r[4 * c + 2] += p.z;
        r[4 * c + 3] += p.w;
      }
    } else {
#pragma unroll
      for (int c = 0; c < NQ / 2; ++c) {
        const float2 p = *reinterpret_cast<const float2*>(src + 2 * c);
        r[2 * c] += p.x;
        r[2 * c + 1] += p.y;
      }
    }
  }

  // Per-antenna sums over all K users of |W|^2.  Afterwards the lane holds the
  // totals r[j], j < NS / 4, of columns i0 + j (column i = 2s + h <-> antenna
  // 8s + 2q + h); returns i0.  par selects the partial buffer (alternating
  // between consecutive calls, so one barrier per call suffices).
  __device__ __forceinline__ static int colsum(const Lane& L, float* np, int par, const WT& w,
                                               float (&r)[NQ]) {
    float v[2 * NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) {
      v[2 * s] = fmaf(w[s][0], w[s][0], w[s][2] * w[s][2]);
      v[2 * s + 1] = fmaf(w[s][1], w[s][1], w[s][3] * w[s][3]);
    }
    const int b2 = (L.g >> 2) & 1, b1 = (L.g >> 1) & 1, b0 = L.g & 1;
    rs_step<NS>(v, b2, 16);
    rs_step<NS / 2>(v, b1, 8);
    rs_step<NS / 4>(v, b0, 4);
    const int i0 = b2 * NS + b1 * (NS / 2) + b0 * (NS / 4);
    st_nq(np + ((par * KW + L.w) * 4 + L.q) * C::NPR + i0, v);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < NQ; ++j) r[j] = 0.f;
#pragma unroll
    for (int ww = 0; ww < KW; ++ww) add_nq(np + ((par * KW + ww) * 4 + L.q) * C::NPR + i0, r);
    return i0;
  }

  // Group soft threshold with tau on all antennas.
  __device__ __forceinline__ static void shrink(const Lane& L, float* np, float* fb, int par,
                                                float tau, WT& w) {
    float r[NQ];
    const int i0 = colsum(L, np, par, w, r);
    const float tau2 = tau * tau;
    float* fw = fb + (L.w * 4 + L.q) * C::NPR;
    float f[NQ];
#pragma unroll
    for (int j = 0; j < NQ; ++j) f[j] = (r[j] > tau2) ? (1.f - tau * rsqrtf(r[j])) : 0.f;
    st_nq(fw + i0, f);
    __syncwarp();
#pragma unroll
    for (int c = 0; c < NS / 2; ++c) {
      const float4 f = *reinterpret_cast<const float4*>(fw + 4 * c);  // columns 4c .. 4c + 3
      w[2 * c][0] *= f.x;
      w[2 * c][2] *= f.x;
      w[2 * c][1] *= f.y;
      w[2 * c][3] *= f.y;
      w[2 * c + 1][0] *= f.z;
      w[2 * c + 1][2] *= f.z;
      w[2 * c + 1][1] *= f.w;
      w[2 * c + 1][3] *= f.w;
    }
    __syncwarp();
  }

  // ------------------------------------------------------------------ setup
  // In-place equilibrated Gauss-Jordan inverse of E = G^T (natural, in Es) over
  // the CTA; pivot row / column staged in rowp / colp.  On success Es = G^{-T}.
  template <int NTX = NT>
  __device__ static bool gj_fp32(const Lane& L, float2* Es, float* dsc, float2* rowp, float2* colp,
                                 float cond_thr) {
    if (L.tid < KB) dsc[L.tid] = rsqrtf(Es[L.tid * KB + L.tid].x);
    __syncthreads();
    for (int idx = L.tid; idx < KB * KB; idx += NTX) {
      const float sc = dsc[idx / KB] * dsc[idx % KB];
      const float2 v = Es[idx];
      Es[idx] = make_float2(v.x * sc, v.y * sc);
    }
    bool fail = false;
    float dmin = FLT_MAX, dmax = 0.f;
#pragma unroll 1
    for (int p = 0; p < KB; ++p) {
      __syncthreads();
      if (L.tid < KB) {
        rowp[L.tid] = Es[p * KB + L.tid];
        colp[L.tid] = Es[L.tid * KB + p];
      }
      __syncthreads();
      const float d = rowp[p].x;
      fail |= !(d > 0.f) || !(d < FLT_MAX);
      dmin = fminf(dmin, d);
      dmax = fmaxf(dmax, d);
      const float inv = rcp_nr(d);
      for (int idx = L.tid; idx < KB * KB; idx += NTX) {
        const int i = idx / KB, j = idx % KB;
        float2 v;
        if (i == p && j == p) {
          v = make_float2(inv, 0.f);
        } else if (i == p) {
          const float2 a = rowp[j];
          v = make_float2(a.x * inv, a.y * inv);
        } else if (j == p) {
          const float2 a = colp[i];
          v = make_float2(-a.x * inv, -a.y * inv);
        } else {
          const float2 a = colp[i], b = rowp[j];
          const float tr = a.x * inv, ti = a.y * inv;
          v = Es[idx];
          v.x -= tr * b.x - ti * b.y;
          v.y -= tr * b.y + ti * b.x;
        }
        Es[idx] = v;
      }
    }
    __syncthreads();
    const bool ok = !fail && !(dmax > cond_thr * dmin);
    if (ok) {
      for (int idx = L.tid; idx < KB * KB; idx += NTX) {
        const float sc = dsc[idx / KB] * dsc[idx % KB];
        const float2 v = Es[idx];
        Es[idx] = make_float2(v.x * sc, v.y * sc);
      }
    }
    __syncthreads();
    return ok;
  }

  // FP64 path: A = G^T from the raw channel in FP64, Gauss-Jordan in FP64 (no
  // equilibration; a pivot below 1e-12 of its Gram diagonal means rank(H) < K),
  // Es = G^{-T} rounded once.  Returns the instance flags.
  __device__ static int gj_fp64(const Lane& L, int K, const float2* Hs, float2* Es, double2* A,
                                double2* rowp, double2* colp, double* orig) {
    for (int idx = L.tid; idx < KB * KB; idx += NT) {
      const int i = idx / KB, j = idx % KB;
      if (j > i) continue;
      double sr = 0.0, si = 0.0;  // sum_m conj(H_im) H_jm
      for (int m = 0; m < MB; ++m) {
        const float2 x = Hs[i * RSF + m], y = Hs[j * RSF + m];
        sr += (double)x.x * y.x + (double)x.y * y.y;
        si += (double)x.x * y.y - (double)x.y * y.x;
      }
      A[i * KB + j] = make_double2(sr, si);
      A[j * KB + i] = make_double2(sr, -si);
    }
    __syncthreads();
    if (L.tid >= K && L.tid < KB) A[L.tid * KB + L.tid] = make_double2(1.0, 0.0);  // padded users
    __syncthreads();
    if (L.tid < KB) orig[L.tid] = A[L.tid * KB + L.tid].x;
    int fl = PRECODE_F_FP64_CHOL;
    bool singular = false;
#pragma unroll 1
    for (int p = 0; p < KB; ++p) {
      __syncthreads();
      if (L.tid < KB) {
        rowp[L.tid] = A[p * KB + L.tid];
        colp[L.tid] = A[L.tid * KB + p];
      }
      __syncthreads();
      const double d = rowp[p].x;
      if (!(d > 1e-12 * orig[p]) || !(d < DBL_MAX)) {
        singular = true;
        break;
      }
      const double inv = 1.0 / d;
      for (int idx = L.tid; idx < KB * KB; idx += NT) {
        const int i = idx / KB, j = idx % KB;
        double2 v;
        if (i == p && j == p) {
          v = make_double2(inv, 0.0);
        } else if (i == p) {
          const double2 a = rowp[j];
          v = make_double2(a.x * inv, a.y * inv);
        } else if (j == p) {
          const double2 a = colp[i];
          v = make_double2(-a.x * inv, -a.y * inv);
        } else {
          const double2 a = colp[i], b = rowp[j];
          const double tr = a.x * inv, ti = a.y * inv;
          v = A[idx];
          v.x -= tr * b.x - ti * b.y;
          v.y -= tr * b.y + ti * b.x;
        }
        A[idx] = v;
      }
    }
    __syncthreads();
    if (singular) {
      for (int k = 0; k < KB; ++k)
        if (!(orig[k] < DBL_MAX) || orig[k] != orig[k]) fl |= PRECODE_F_NONFINITE;
      return fl | PRECODE_F_SINGULAR;
    }
    for (int idx = L.tid; idx < KB * KB; idx += NT)
      Es[idx] = make_float2((float)A[idx].x, (float)A[idx].y);
    __syncthreads();
    return fl;
  }

  // FP64 path in an orthonormal basis of the channel's row space.  With
  // G = H H^H = L D L^H (FP64; a pivot below 1e-12 of its Gram diagonal means
  // rank(H) < K) the rows of U = D^{-1/2} L^{-1} H are orthonormal and span H's
  // row space, and H W^T = S becomes U W^T = S~ with S~ = D^{-1/2} L^{-1} S.  The
  // projection onto it is X - (X U^T - S~^T) conj(U): the layers' map with U in
  // place of the channel, the identity in place of G^{-T} and S~^T in place of S.
  // Rounding U to FP32 perturbs that orthogonal projector by O(u) at any
  // conditioning, while G^{-T} rounded to FP32 perturbs the projector by
  // O(u cond G), which the layers amplify once u cond G nears 1.  Writes U over
  // the channel rows (in place, one thread per antenna column), S~^T into Es
  // (natural [KB][KB]) and, unless gf is null, the identity's B fragments into gf.  Padded users
  // (K <= k < KB) have zero channel rows and targets and get a unit pivot, so
  // their rows of U and of S~ stay zero.  Returns the instance flags.
  template <int NTX = NT>
  __device__ static int basis_fp64(const Lane& L, int K, float2* Hs, float2* Es, float4* gf,
                                   double2* A, double* piv, double* ipv, double* orig,
                                   const float* tks) {
    for (int idx = L.tid; idx < KB * KB; idx += NTX) {
      const int i = idx / KB, j = idx % KB;
      if (j > i) continue;
      double sr = 0.0, si = 0.0;  // sum_m H_im conj(H_jm)
      for (int m = 0; m < MB; ++m) {
        const float2 x = Hs[i * RSF + m], y = Hs[j * RSF + m];
        sr += (double)x.x * y.x + (double)x.y * y.y;
        si += (double)x.y * y.x - (double)x.x * y.y;
      }
      A[i * KB + j] = make_double2(sr, si);
    }
    __syncthreads();
    if (L.tid >= K && L.tid < KB) A[L.tid * KB + L.tid] = make_double2(1.0, 0.0);  // padded users
    __syncthreads();
    if (L.tid < KB) orig[L.tid] = A[L.tid * KB + L.tid].x;
    __syncthreads();
    int fl = PRECODE_F_FP64_CHOL;
    bool singular = false;
#pragma unroll 1
    for (int p = 0; p < KB; ++p) {  // right-looking LDL^H on the lower triangle
      const double d = A[p * KB + p].x;
      if (!(d > 1e-12 * orig[p]) || !(d < DBL_MAX)) {
        singular = true;
        break;
      }
      const double inv = 1.0 / d;
      const int R = KB - 1 - p;
      for (int idx = L.tid; idx < R * R; idx += NTX) {
        const int i = p + 1 + idx / R, l = p + 1 + idx % R;
        if (l > i) continue;
        const double2 aip = A[i * KB + p], alp = A[l * KB + p];
        const double ar = aip.x * inv, ai = aip.y * inv;
        double2 v = A[i * KB + l];
        v.x -= ar * alp.x + ai * alp.y;  // a conj(b)
        v.y -= ai * alp.x - ar * alp.y;
        A[i * KB + l] = v;
      }
      __syncthreads();
    }
    if (singular) {
      for (int k = 0; k < KB; ++k)
        if (!(orig[k] < DBL_MAX) || orig[k] != orig[k]) fl |= PRECODE_F_NONFINITE;
      __syncthreads();
      return fl | PRECODE_F_SINGULAR;
    }
    if (L.tid < KB) {
      piv[L.tid] = A[L.tid * KB + L.tid].x;
      ipv[L.tid] = 1.0 / A[L.tid * KB + L.tid].x;
    }
    __syncthreads();
    // U by forward substitution L Y = H, column by column in FP64, then D^{-1/2}
#pragma unroll 1
    for (int m = L.tid; m < MB; m += NTX) {
      double yr[KB], yi[KB];
#pragma unroll 1
      for (int i = 0; i < KB; ++i) {
        const float2 h = Hs[i * RSF + m];
        double sr = h.x, si = h.y;
#pragma unroll 1
        for (int p = 0; p < i; ++p) {
          const double2 a = A[i * KB + p];  // L[i][p] d_p
          const double lr = a.x * ipv[p], li = a.y * ipv[p];
          sr -= lr * yr[p] - li * yi[p];
          si -= lr * yi[p] + li * yr[p];
        }
        yr[i] = sr;
        yi[i] = si;
      }
#pragma unroll 1
      for (int i = 0; i < KB; ++i) {
        const double sc = 1.0 / sqrt(piv[i]);
        Hs[i * RSF + m] = make_float2((float)(yr[i] * sc), (float)(yi[i] * sc));
      }
    }
    // S~^T[k][i] = S~[i][k]: forward substitution of t_k e_k
#pragma unroll 1
    for (int k = L.tid; k < KB; k += NTX) {
      double yr[KB], yi[KB];
#pragma unroll 1
      for (int i = 0; i < KB; ++i) {
        double sr = (i == k) ? (double)tks[k] : 0.0, si = 0.0;
#pragma unroll 1
        for (int p = k; p < i; ++p) {
          const double2 a = A[i * KB + p];
          const double lr = a.x * ipv[p], li = a.y * ipv[p];
          sr -= lr * yr[p] - li * yi[p];
          si -= lr * yi[p] + li * yr[p];
        }
        yr[i] = sr;
        yi[i] = si;
      }
#pragma unroll 1
      for (int i = 0; i < KB; ++i) {
        const double sc = 1.0 / sqrt(piv[i]);
        Es[k * KB + i] = i < k ? make_float2(0.f, 0.f)
                               : make_float2((float)(yr[i] * sc), (float)(yi[i] * sc));
      }
    }
    __syncthreads();  // the FP64 scratch is read out: the identity's fragments go over it
    for (int idx = L.tid; gf && idx < KW * KW * 32; idx += NTX) {
      const int kt = idx / (KW * 32), cp = (idx / 32) % KW, ln = idx % 32;
      const int gg = ln >> 2, qq = ln & 3;
      gf[idx] = make_float4(8 * kt + 2 * qq == 8 * cp + gg ? 1.f : 0.f,
                            8 * kt + 2 * qq + 1 == 8 * cp + gg ? 1.f : 0.f, 0.f, 0.f);
    }
    __syncthreads();
    return fl;
  }

  // The instance's channel rows again from global memory (over U, after the
  // layers of an instance solved in the orthonormal basis), each row times
  // rs[k] when rs is given (a power of two: exact).
  __device__ static void reload_channel(const Lane& L, int K, const float2* Hg, float2* Hs,
                                        const float* rs = nullptr) {
    for (int idx = L.tid; idx < K * (MB / 2); idx += NT) {
      const int k = idx / (MB / 2), m2 = idx % (MB / 2);
      float4 v = *reinterpret_cast<const float4*>(Hg + k * MB + 2 * m2);
      if (rs) {
        const float f = rs[k];
        v = make_float4(f * v.x, f * v.y, f * v.z, f * v.w);
      }
      *reinterpret_cast<float4*>(Hs + k * RSF + 2 * m2) = v;
    }
    __syncthreads();
  }

  // ---------------------------------------------------------------- kernel
  __device__ static void run(const SolveArgs& A) {
    extern __shared__ __align__(16) unsigned char smem[];
    Lane L;
    L.tid = threadIdx.x;
    L.w = L.tid >> 5;
    L.lane = L.tid & 31;
    L.g = L.lane >> 2;
    L.q = L.lane & 3;
    float2* const Hs = reinterpret_cast<float2*>(smem);
    float2* const Es = reinterpret_cast<float2*>(smem + C::OFF_E);
    float4* const gf = reinterpret_cast<float4*>(smem + C::OFF_GF);
    float* const np = reinterpret_cast<float*>(smem + C::OFF_NP);
    float* const fb = reinterpret_cast<float*>(smem + C::OFF_FB);
    float4* const ft = reinterpret_cast<float4*>(smem + C::OFF_FT) + L.w * KW * 32;
    double2* const A64 = reinterpret_cast<double2*>(smem + C::OFF_X);
    double2* const r64 = reinterpret_cast<double2*>(smem + C::OFF_S64);
    double2* const c64 = r64 + KB;
    double* const o64 = reinterpret_cast<double*>(c64 + KB);
    float* const tks = reinterpret_cast<float*>(smem + C::OFF_SC);
    float* const dsc = tks + KB;
    float2* const rowp = reinterpret_cast<float2*>(dsc + KB);
    float2* const colp = rowp + KB;
    int* const misc = reinterpret_cast<int*>(colp + KB);
    float* const wred = reinterpret_cast<float*>(misc + 8);
    uint64_t* const bar = reinterpret_cast<uint64_t*>(smem + C::OFF_BAR);
    if (L.tid == 0) mbar_init(bar, 1);
    fence_mbar_init();
    __syncthreads();

    uint32_t phase = 0;
    int par = 0;
    const int64_t n_inst = A.tbl ? (int64_t)(*A.count) : A.B;
    auto locate = [&](int64_t it, int64_t& inst, int64_t& h_off, int64_t& w_off, int64_t& t_off,
                      int& K) {
      if (A.tbl) {
        inst = A.index[it];
        const InstDesc d = A.tbl[inst];
        h_off = d.h_off;
        w_off = d.w_off;
        t_off = d.t_off;
        K = d.K;
      } else {
        inst = it;
        K = A.K;
        h_off = it * (int64_t)(K * MB);
        w_off = h_off;
        t_off = it * A.t_stride;
      }
    };
    // the channel's K rows, each to its padded shared-memory row
    auto issue_copy = [&](int64_t it) {
      if (L.tid != 0 || it >= n_inst || (A.opts & OPT_STALL_COPY)) return;
      int64_t inst, h_off, w_off, t_off;
      int K;
      locate(it, inst, h_off, w_off, t_off, K);
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, K * MB * 8);
      for (int k = 0; k < K; ++k) bulk_g2s(Hs + k * RSF, A.H + h_off + k * MB, MB * 8, bar);
    };
    issue_copy(blockIdx.x);
    WT w;
#pragma unroll 1
    for (int64_t it = blockIdx.x; it < n_inst; it += gridDim.x) {
      int64_t inst, h_off, w_off, t_off;
      int K;
      locate(it, inst, h_off, w_off, t_off, K);
      if (L.tid < KB) tks[L.tid] = L.tid < K ? A.t[t_off + L.tid] : 0.f;
      if (L.tid == 0) misc[0] = mbar_wait_bounded(bar, phase, copy_wait_ns(A)) ? 1 : 0;
      __syncthreads();
      if (misc[0] == 0) {
        if (L.tid == 0) {
          atomicAdd(A.err, 1ull);
          if (A.flags) A.flags[inst] = PRECODE_F_TIMEOUT;
          misc[1] = mbar_wait_bounded(bar, phase, copy_wait_ns(A)) ? 1 : 0;
        }
        __syncthreads();
        if (misc[1] == 0) return;
        phase ^= 1u;
        __syncthreads();
        issue_copy(it + gridDim.x);
        continue;
      }
      if (L.tid != 0) mbar_wait_bounded(bar, phase, copy_wait_ns(A));  // completed: returns at once
      phase ^= 1u;
      if (K < KB) {  // padded users: zero channel rows
        for (int idx = L.tid; idx < (KB - K) * MB; idx += NT)
          Hs[(K + idx / MB) * RSF + idx % MB] = make_float2(0.f, 0.f);
        __syncthreads();
      }

      // ---- setup
      int fl = 0;
      float invL = 1.f;
      const bool need_gram = (MODE == kModeProj) || (A.opts & OPT_STEP_NORMALISED);
      if (need_gram) {
#pragma unroll 1
        for (int ct = 0; ct < KW; ++ct) {  // G^T rows 8w .. 8w + 7
          float e[4];
          e_tile<true>(L, Hs, w, ct, e);
          float2* row = Es + (8 * L.w + L.g) * KB + 8 * ct + 2 * L.q;
          *reinterpret_cast<float4*>(row) = make_float4(e[0], e[2], e[1], e[3]);
        }
        __syncthreads();
        if (MODE == kModeProj && K < KB) {  // padded users: unit Gram diagonal
          if (L.tid >= K && L.tid < KB) Es[L.tid * KB + L.tid] = make_float2(1.f, 0.f);
          __syncthreads();
        }
      }
      bool singular = false, basis = false;
      if constexpr (MODE == kModeProj) {
        if (!gj_fp32(L, Es, dsc, rowp, colp, A.cond_thr)) {
          fl = basis_fp64(L, K, Hs, Es, gf, A64, reinterpret_cast<double*>(r64),
                          reinterpret_cast<double*>(c64), o64, tks);
          singular = (fl & PRECODE_F_SINGULAR) != 0;
          basis = !singular;
        }
        if (!singular) {
          // G^{-T} as B fragments (the basis path wrote the identity's), then
          // W^(0) = S G^{-T} conj(H) = 0 - F0 conj(H) with F0 = -S G^{-T} (the warp's
          // rows; S~^T conj(U) with F0 = -S~^T in the basis)
          if (!basis) {
            for (int idx = L.tid; idx < KW * KW * 32; idx += NT) {
              const int kt = idx / (KW * 32), cp = (idx / 32) % KW, ln = idx % 32;
              const int gg = ln >> 2, qq = ln & 3;
              const float2 m0 = Es[(8 * kt + 2 * qq) * KB + 8 * cp + gg];
              const float2 m1 = Es[(8 * kt + 2 * qq + 1) * KB + 8 * cp + gg];
              gf[idx] = make_float4(m0.x, m1.x, m0.y, m1.y);
            }
          }
          const float tg = basis ? 1.f : tks[8 * L.w + L.g];
#pragma unroll 1
          for (int kt = 0; kt < KW; ++kt) {
            const float4 v =
                *reinterpret_cast<const float4*>(Es + (8 * L.w + L.g) * KB + 8 * kt + 2 * L.q);
            ft[kt * 32 + L.lane] = make_float4(-tg * v.x, -tg * v.z, -tg * v.y, -tg * v.w);
          }
          __syncthreads();
#pragma unroll
          for (int s = 0; s < NS; ++s)
#pragma unroll
            for (int k = 0; k < 4; ++k) w[s][k] = 0.f;
          update(L, Hs, ft, w);
        }
      } else {
        if (A.opts & OPT_STEP_NORMALISED) {  // 1 / Gershgorin bound max_k sum_j |G_kj|
          if (L.tid < K) {
            float sacc = 0.f;
            for (int j = 0; j < K; ++j) {
              const float2 v = Es[L.tid * KB + j];
              sacc += sqrtf(v.x * v.x + v.y * v.y);
            }
            dsc[L.tid] = sacc;
          }
          __syncthreads();
          float Lg = 0.f;
          for (int k = 0; k < K; ++k) Lg = fmaxf(Lg, dsc[k]);
          invL = 1.f / Lg;
        }
        const float2* hr = Hs + (8 * L.w + L.g) * RSF + 2 * L.q;  // W^(0) = conj(H)
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          const float4 v = *reinterpret_cast<const float4*>(hr + 8 * s);
          w[s][0] = v.x;
          w[s][1] = v.z;
          w[s][2] = -v.y;
          w[s][3] = -v.w;
        }
      }

      // ---- layers
      const int T = A.T;
      float rss = 0.f;
      if (!singular) {
#pragma unroll 1
        for (int l = 0; l < T; ++l) {
          if constexpr (MODE == kModeProj) {
            shrink(L, np, fb, par, fmaxf(__ldg(A.step + l), 0.f), w);
            par ^= 1;
            residual_f(L, Hs, gf, tks, 1.f, w, ft, basis ? Es : nullptr);
            update(L, Hs, ft, w);
          } else {
            const float eta = __ldg(A.step + l) * invL;
            residual_f(L, Hs, gf, tks, eta, w, ft);
            update(L, Hs, ft, w);
            shrink(L, np, fb, par, fmaxf(fmaxf(__ldg(A.lam + l), 0.f) * eta, 0.f), w);
            par ^= 1;
          }
        }
        if (A.resid) {
          if (basis) {  // against the channel itself
            __syncthreads();
            reload_channel(L, K, A.H + h_off, Hs);
          }
          rss = residual_ss(L, Hs, tks, w);
#pragma unroll
          for (int msk = 1; msk < 32; msk <<= 1) rss += __shfl_xor_sync(FULL, rss, msk);
        }
      } else {
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int k = 0; k < 4; ++k) w[s][k] = 0.f;
        if (L.w == 0 && L.lane == 0)
          for (int k = 0; k < KB; ++k) rss += tks[k] * tks[k];
      }
      if (L.lane == 0) wred[L.w] = rss;

      // ---- objective (column norms over all users), then the channel buffer is
      // free: next copy, W write-back, scalars
      float r[NQ];
      colsum(L, np, par, w, r);
      par ^= 1;
      float o = 0.f;
#pragma unroll
      for (int j = 0; j < NQ; ++j) o += sqrtf(r[j]);
#pragma unroll
      for (int msk = 1; msk < 32; msk <<= 1) o += __shfl_xor_sync(FULL, o, msk);
      __syncthreads();  // every warp is done with the channel and wred is complete
      issue_copy(it + gridDim.x);
      if (8 * L.w + L.g < K) {
        float2* const Wg = A.W + w_off + (8 * L.w + L.g) * MB + 2 * L.q;
#pragma unroll
        for (int s = 0; s < NS; ++s)
          *reinterpret_cast<float4*>(Wg + 8 * s) = make_float4(w[s][0], w[s][2], w[s][1], w[s][3]);
      }
      if (L.tid == 0) {
        float rs = 0.f;
        for (int k = 0; k < KW; ++k) rs += wred[k];
        if (!(o < FLT_MAX) || !(rs < FLT_MAX)) fl |= PRECODE_F_NONFINITE;
        if (A.obj) A.obj[inst] = o;
        if (A.resid) A.resid[inst] = sqrtf(rs);
        if (A.flags) A.flags[inst] = fl;
      }
    }
  }
};

template <int MODE, int KW, int MB, int MINB>
__global__ void __launch_bounds__(KW * 32, MINB) solve_tcw_kernel(SolveArgs A) {
  SolveTCW<MODE, KW, MB>::run(A);
}

}  // namespace precode
