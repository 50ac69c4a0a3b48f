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
// column norms of the shrink reduce over the 8 lanes of a column (through shared
// memory).
#pragma once

#include "solve.cuh"
#include "tf32mma.cuh"

namespace precode {

template <int MODE, int NW, bool DB>
struct SolveTC : SolveKernel<MODE, 8, 64, 4, 8, 8, true, NW, true, DB> {
  using Base = SolveKernel<MODE, 8, 64, 4, 8, 8, true, NW, true, DB>;
  using C = typename Base::C;
  using Ctx = typename Base::Ctx;
  static constexpr int KB = 8, MB = 64;
  // antenna tiles per update batch (4 independent MMA chains; 2 keeps the paper
  // layer's build inside its 128 registers)
  static constexpr int UG = MODE == kModeProj ? 4 : 2;
  static constexpr int NHB = C::NHB;
  // Per-warp shared memory, two overlaid phases (bytes):
  //   setup : H (raw channel) | Q / FP64 scratch | Gauss-Jordan buffers | Gram
  //   layers: H hi parts (in place) | X fragments hi/lo | H lo parts | norm partials | factors
  //   both  : t, scalars, copy barriers (and the second channel buffer with prefetch)
  static constexpr int H_BYTES = KB * MB * 8;
  static constexpr int OFF_Q = H_BYTES;                       // setup
  static constexpr int OFF_RED = OFF_Q + KB * MB * 8;         // setup
  static constexpr int OFF_E = OFF_RED + C::RED_BYTES;        // setup
  // Without prefetch the layers read H pre-split (hi in place, lo beside it);
  // with prefetch they split it on the fly, which leaves room for the second
  // channel buffer at the same occupancy.
  static constexpr bool PRE = !DB;
  static constexpr int OFF_XF = H_BYTES;                      // layers, 8 KB
  static constexpr int OFF_LO = OFF_XF + 8192;                // layers, 4 KB (PRE)
  static constexpr int OFF_NB = OFF_LO + (PRE ? H_BYTES : 0); // layers, 2 KB
  static constexpr int OFF_FB = OFF_NB + 2048;                // layers, 256 B
  static constexpr int OFF_ST = OFF_FB + 256;                 // S~^T of the FP64 path, 512 B
  static constexpr int OFF_SC = OFF_ST + KB * KB * 8;
  static constexpr int OFF_BAR = OFF_SC + C::SC_BYTES;
  static constexpr int OFF_H1 = align_up(OFF_BAR + 8 * NHB, 16);
  static constexpr int GROUP_STRIDE = OFF_H1 + (DB ? H_BYTES : 0);
  static constexpr int SMEM_BYTES = C::GROUPS * GROUP_STRIDE;
  static_assert(OFF_E + KB * KB * 8 <= OFF_ST, "setup buffers stay clear of S~^T and the scalars");
  static_assert(C::GROUPS == NW, "one instance per warp");

  struct Lane {
    int g, q, lane;
  };
  // W in MMA accumulator order: w[s] = (Re W[g][8s+2q], Re W[g][8s+2q+1],
  //                                     Im W[g][8s+2q], Im W[g][8s+2q+1])
  using WT = float[8][4];

  // Column (antenna) sums over the 8 users of |W|^2: each lane stores its 16
  // partial squares, then lane (rq, rs) = (lane % 4, lane / 4) adds up antennas
  // 8 rs + 2 rq + {0, 1} over the users.  Chunks of 4 floats are XOR-swizzled so
  // that both the 128-bit stores and the 64-bit column reads are conflict free.
  __device__ __forceinline__ static int nb_swz(int writer) {
    const int b = writer >> 1;
    return ((b & 1) << 1) | ((b >> 1) & 1);
  }
  __device__ __forceinline__ static float2 colsum(const Lane& L, float* nb, const WT& w) {
    const int sw = nb_swz(L.lane);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float4 p;
      p.x = fmaf(w[2 * j][0], w[2 * j][0], w[2 * j][2] * w[2 * j][2]);
      p.y = fmaf(w[2 * j][1], w[2 * j][1], w[2 * j][3] * w[2 * j][3]);
      p.z = fmaf(w[2 * j + 1][0], w[2 * j + 1][0], w[2 * j + 1][2] * w[2 * j + 1][2]);
      p.w = fmaf(w[2 * j + 1][1], w[2 * j + 1][1], w[2 * j + 1][3] * w[2 * j + 1][3]);
      *reinterpret_cast<float4*>(nb + L.lane * 16 + 4 * (j ^ sw)) = p;
    }
    __syncwarp();
    const int rq = L.lane & 3, rs = L.lane >> 2;
    float2 a = make_float2(0.f, 0.f);
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int wr = 4 * g + rq;
      const float2 v =
          *reinterpret_cast<const float2*>(nb + wr * 16 + 4 * ((rs >> 1) ^ nb_swz(wr)) + (rs & 1) * 2);
      a.x += v.x;
      a.y += v.y;
    }
    return a;
  }

  // Group soft threshold with the column sums of colsum: the reading lane forms
  // the factors of its two antennas, every lane then scales its own entries.
  __device__ __forceinline__ static void shrink(const Lane& L, float* fb, float2 r2, float tau,
                                                WT& w) {
    const float tau2 = tau * tau;
    const float f0 = (r2.x > tau2) ? (1.f - tau * rsqrtf(r2.x)) : 0.f;
    const float f1 = (r2.y > tau2) ? (1.f - tau * rsqrtf(r2.y)) : 0.f;
    const int rq = L.lane & 3, rs = L.lane >> 2;
    *reinterpret_cast<float2*>(fb + rq * 16 + 4 * ((rs >> 1) ^ (rq & 2)) + (rs & 1) * 2) =
        make_float2(f0, f1);
    __syncwarp();
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float4 f = *reinterpret_cast<const float4*>(fb + L.q * 16 + 4 * (j ^ (L.q & 2)));
      w[2 * j][0] *= f.x;
      w[2 * j][2] *= f.x;
      w[2 * j][1] *= f.y;
      w[2 * j][3] *= f.y;
      w[2 * j + 1][0] *= f.z;
      w[2 * j + 1][2] *= f.z;
      w[2 * j + 1][1] *= f.w;
      w[2 * j + 1][3] *= f.w;
    }
  }

  // E = W H^T (minus S on the diagonal when sub_s): returns the lane's fragment
  // e = (E_re[g][2q], E_re[g][2q+1], E_im[g][2q], E_im[g][2q+1]).  Every MMA
  // takes the same A quad (Re W, Im W rows); products with Re H go to ar, with
  // Im H to ai, so that
  //   E_re = [ar]_row g - [ai]_row g+8,   E_im = [ai]_row g + [ar]_row g+8
  // (no negated or permuted copies of W).  Two blocks of 8 antennas at a time,
  // term by term (lo terms first).
  // PRE: H comes pre-split, hi / lo fragments (Hr0, Hr1, Hi0, Hi1) at [s][lane];
  // otherwise it is read from the raw channel and split here.
  template <bool PRE>
  __device__ __forceinline__ static void residual(const Lane& L, const float2* Hs, const float4* hhi,
                                                  const float4* hlo, const WT& w, const float* tks,
                                                  bool sub_s, float (&e)[4]) {
    float ar[2][4], ai[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) ar[i][k] = ai[i][k] = 0.f;
#pragma unroll
    for (int s0 = 0; s0 < 8; s0 += 2) {
      uint32_t bh[2][4], bl[2][4], ah[2][4], al[2][4];  // [block][hr0 hr1 hi0 hi1 / r0 i0 r1 i1]
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int s = s0 + u;
        if constexpr (PRE) {
          const float4 hh = hhi[s * 32 + L.lane], hl = hlo[s * 32 + L.lane];
          bh[u][0] = __float_as_uint(hh.x);
          bh[u][1] = __float_as_uint(hh.y);
          bh[u][2] = __float_as_uint(hh.z);
          bh[u][3] = __float_as_uint(hh.w);
          bl[u][0] = __float_as_uint(hl.x);
          bl[u][1] = __float_as_uint(hl.y);
          bl[u][2] = __float_as_uint(hl.z);
          bl[u][3] = __float_as_uint(hl.w);
        } else {
          const float4 hv = *reinterpret_cast<const float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
          split_tf32(hv.x, bh[u][0], bl[u][0]);
          split_tf32(hv.z, bh[u][1], bl[u][1]);
          split_tf32(hv.y, bh[u][2], bl[u][2]);
          split_tf32(hv.w, bh[u][3], bl[u][3]);
        }
        split_tf32(w[s][0], ah[u][0], al[u][0]);  // Re W, h = 0
        split_tf32(w[s][2], ah[u][1], al[u][1]);  // Im W, h = 0
        split_tf32(w[s][1], ah[u][2], al[u][2]);  // Re W, h = 1
        split_tf32(w[s][3], ah[u][3], al[u][3]);  // Im W, h = 1
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mma_tf32(ar[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bl[u][0], bl[u][1]);
        mma_tf32(ai[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bl[u][2], bl[u][3]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mma_tf32(ar[u], al[u][0], al[u][1], al[u][2], al[u][3], bh[u][0], bh[u][1]);
        mma_tf32(ai[u], al[u][0], al[u][1], al[u][2], al[u][3], bh[u][2], bh[u][3]);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mma_tf32(ar[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bh[u][0], bh[u][1]);
        mma_tf32(ai[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bh[u][2], bh[u][3]);
      }
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
    // -A: k-step 0 = (-c0, -c2, -c1, -c3), k-step 1 = (c2, -c0, c3, -c1)
    const uint32_t n0h = neg_bits(c0h), n1h = neg_bits(c1h), n2h = neg_bits(c2h),
                   n3h = neg_bits(c3h);
    const uint32_t n0l = neg_bits(c0l), n1l = neg_bits(c1l), n2l = neg_bits(c2l),
                   n3l = neg_bits(c3l);
#pragma unroll
    for (int nt0 = 0; nt0 < 8; nt0 += UG) {
      float4 xh[UG], xl[UG];
      float d[UG][4];  // the product from zero, added to W rounded (see SolveTCH::update_h)
#pragma unroll
      for (int u = 0; u < UG; ++u) {
#pragma unroll
        for (int k = 0; k < 4; ++k) d[u][k] = 0.f;
        xh[u] = xf[((nt0 + u) * 2 + 0) * 32 + L.lane];
        xl[u] = xf[((nt0 + u) * 2 + 1) * 32 + L.lane];
      }
      if constexpr (MODE == kModeProj) {  // into W directly (see SolveTCH::update_h)
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(w[nt0 + u], n0h, n2h, n1h, n3h, __float_as_uint(xl[u].x), __float_as_uint(xl[u].y));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(w[nt0 + u], n0l, n2l, n1l, n3l, __float_as_uint(xh[u].x), __float_as_uint(xh[u].y));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(w[nt0 + u], c2h, n0h, c3h, n1h, __float_as_uint(xl[u].z), __float_as_uint(xl[u].w));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(w[nt0 + u], c2l, n0l, c3l, n1l, __float_as_uint(xh[u].z), __float_as_uint(xh[u].w));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(w[nt0 + u], n0h, n2h, n1h, n3h, __float_as_uint(xh[u].x), __float_as_uint(xh[u].y));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(w[nt0 + u], c2h, n0h, c3h, n1h, __float_as_uint(xh[u].z), __float_as_uint(xh[u].w));
      } else {
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(d[u], n0h, n2h, n1h, n3h, __float_as_uint(xl[u].x), __float_as_uint(xl[u].y));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(d[u], n0l, n2l, n1l, n3l, __float_as_uint(xh[u].x), __float_as_uint(xh[u].y));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(d[u], c2h, n0h, c3h, n1h, __float_as_uint(xl[u].z), __float_as_uint(xl[u].w));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(d[u], c2l, n0l, c3l, n1l, __float_as_uint(xh[u].z), __float_as_uint(xh[u].w));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(d[u], n0h, n2h, n1h, n3h, __float_as_uint(xh[u].x), __float_as_uint(xh[u].y));
#pragma unroll
        for (int u = 0; u < UG; ++u)
          mma_tf32(d[u], c2h, n0h, c3h, n1h, __float_as_uint(xh[u].z), __float_as_uint(xh[u].w));
#pragma unroll
        for (int u = 0; u < UG; ++u)
#pragma unroll
          for (int k = 0; k < 4; ++k) w[nt0 + u][k] += d[u][k];
      }
    }
  }

  // Inverse of the Gram matrix from the lane's fragment e of E = G^T (Hermitian,
  // same diagonal and conditioning as G): the equilibrated matrix D E D (D =
  // diag(E)^{-1/2}) is inverted by Gauss-Jordan elimination without pivoting,
  // every lane keeping its own two entries in registers and fetching the pivot
  // row and column by shuffles.  The pivots are the LDL^H pivots, so their
  // spread max/min is the condition estimate.  Returns false (and the caller
  // takes the FP64 path) when a pivot is not positive and finite or the estimate
  // exceeds cond_thr; otherwise gi = the lane's entries (g, 2q), (g, 2q + 1) of
  // G^{-T} = D (D E D)^{-1} D as (re, re, im, im).
  __device__ __forceinline__ static bool gram_inverse(const Lane& L, const float (&e)[4],
                                                      float cond_thr, float (&gi)[4]) {
    constexpr unsigned FULL = 0xffffffffu;
    const float dg_own = (L.g == 2 * L.q) ? e[0] : e[1];  // E[i][i] sits on lane (i, i / 2)
    const float sg = rsqrtf(__shfl_sync(FULL, dg_own, 4 * L.g + (L.g >> 1)));
    const float s0 = rsqrtf(__shfl_sync(FULL, dg_own, 9 * L.q));      // lane (2q, q)
    const float s1 = rsqrtf(__shfl_sync(FULL, dg_own, 9 * L.q + 4));  // lane (2q + 1, q)
    float ar0 = e[0] * (sg * s0), ar1 = e[1] * (sg * s1);
    float ai0 = e[2] * (sg * s0), ai1 = e[3] * (sg * s1);
    bool fail = false;
    float dmin = FLT_MAX, dmax = 0.f;
#pragma unroll
    for (int p = 0; p < KB; ++p) {
      const int own = 4 * L.g + (p >> 1);  // lane holding (g, p)
      const int prow = 4 * p + L.q;        // lane holding (p, 2q), (p, 2q + 1)
      const float d = __shfl_sync(FULL, (p & 1) ? ar1 : ar0, 4 * p + (p >> 1));
      const float pr0 = __shfl_sync(FULL, ar0, prow), pr1 = __shfl_sync(FULL, ar1, prow);
      const float pi0 = __shfl_sync(FULL, ai0, prow), pi1 = __shfl_sync(FULL, ai1, prow);
      const float cr = __shfl_sync(FULL, (p & 1) ? ar1 : ar0, own);
      const float ci = __shfl_sync(FULL, (p & 1) ? ai1 : ai0, own);
      fail |= !(d > 0.f) || !(d < FLT_MAX);
      dmin = fminf(dmin, d);
      dmax = fmaxf(dmax, d);
      const float inv = rcp_nr(d);
      const float tr = cr * inv, ti = ci * inv;  // A[g][p] / d
      // generic entry: a - (A[g][p] / d) A[p][j]
      float n0r = ar0 - (tr * pr0 - ti * pi0), n0i = ai0 - (tr * pi0 + ti * pr0);
      float n1r = ar1 - (tr * pr1 - ti * pi1), n1i = ai1 - (tr * pi1 + ti * pr1);
      const bool rowp = L.g == p, c0p = 2 * L.q == p, c1p = 2 * L.q + 1 == p;
      if (rowp) {  // pivot row: A[p][j] / d
        n0r = pr0 * inv;
        n0i = pi0 * inv;
        n1r = pr1 * inv;
        n1i = pi1 * inv;
      }
      if (c0p) {  // pivot column: -A[i][p] / d, pivot 1 / d
        n0r = rowp ? inv : -tr;
        n0i = rowp ? 0.f : -ti;
      }
      if (c1p) {
        n1r = rowp ? inv : -tr;
        n1i = rowp ? 0.f : -ti;
      }
      ar0 = n0r;
      ar1 = n1r;
      ai0 = n0i;
      ai1 = n1i;
    }
    gi[0] = ar0 * (sg * s0);
    gi[1] = ar1 * (sg * s1);
    gi[2] = ai0 * (sg * s0);
    gi[3] = ai1 * (sg * s1);
    return !fail && !(dmax > cond_thr * dmin);
  }

  // Q = G^{-T} H^* and its transpose as split-TF32 MMAs on the same fragments:
  //   Q   tile nt (rows user g, antennas 8nt + 2q + {0,1}) = G^{-T} conj(H), whose
  //       accumulator is W's own layout, so W^(0) = S Q needs no data movement;
  //   Q^T tile nt = conj(H)^T G^{-1}, whose accumulator is exactly the update's
  //       B fragment (Q[2q][8nt+g], Q[2q+1][8nt+g]), stored split into xf.
  // The A operand of one product is the B operand of the other: the lane's G^{-T}
  // entries gi and the channel entries H[2q][8nt+g], H[2q+1][8nt+g].
  __device__ __forceinline__ static void q_mma(const Lane& L, const float2* Hs, const float (&gi)[4],
                                               float tg, float4* xf, WT& w) {
    uint32_t gr0h, gr0l, gr1h, gr1l, gi0h, gi0l, gi1h, gi1l;
    split_tf32(gi[0], gr0h, gr0l);
    split_tf32(gi[1], gr1h, gr1l);
    split_tf32(gi[2], gi0h, gi0l);
    split_tf32(gi[3], gi1h, gi1l);
    const uint32_t ngi0h = neg_bits(gi0h), ngi0l = neg_bits(gi0l);
    const uint32_t ngi1h = neg_bits(gi1h), ngi1l = neg_bits(gi1l);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      const float2 h0 = Hs[(2 * L.q) * MB + 8 * nt + L.g];
      const float2 h1 = Hs[(2 * L.q + 1) * MB + 8 * nt + L.g];
      uint32_t xr0h, xr0l, xr1h, xr1l, xi0h, xi0l, xi1h, xi1l;  // X = conj(H)
      split_tf32(h0.x, xr0h, xr0l);
      split_tf32(h1.x, xr1h, xr1l);
      split_tf32(-h0.y, xi0h, xi0l);
      split_tf32(-h1.y, xi1h, xi1l);
      const uint32_t nxi0h = neg_bits(xi0h), nxi0l = neg_bits(xi0l);
      const uint32_t nxi1h = neg_bits(xi1h), nxi1l = neg_bits(xi1l);
      float qt[4] = {0.f, 0.f, 0.f, 0.f}, qq[4] = {0.f, 0.f, 0.f, 0.f};
      // Q^T: k-step 0 A = (xr0, xi0, xr1, xi1), B = (gr0, gr1);
      //      k-step 1 A = (-xi0, xr0, -xi1, xr1), B = (gi0, gi1)
      // Q:   k-step 0 A = (gr0, gi0, gr1, gi1), B = (xr0, xr1);
      //      k-step 1 A = (-gi0, gr0, -gi1, gr1), B = (xi0, xi1)
      mma_tf32(qt, xr0h, xi0h, xr1h, xi1h, gr0l, gr1l);
      mma_tf32(qq, gr0h, gi0h, gr1h, gi1h, xr0l, xr1l);
      mma_tf32(qt, xr0l, xi0l, xr1l, xi1l, gr0h, gr1h);
      mma_tf32(qq, gr0l, gi0l, gr1l, gi1l, xr0h, xr1h);
      mma_tf32(qt, nxi0h, xr0h, nxi1h, xr1h, gi0l, gi1l);
      mma_tf32(qq, ngi0h, gr0h, ngi1h, gr1h, xi0l, xi1l);
      mma_tf32(qt, nxi0l, xr0l, nxi1l, xr1l, gi0h, gi1h);
      mma_tf32(qq, ngi0l, gr0l, ngi1l, gr1l, xi0h, xi1h);
      mma_tf32(qt, xr0h, xi0h, xr1h, xi1h, gr0h, gr1h);
      mma_tf32(qq, gr0h, gi0h, gr1h, gi1h, xr0h, xr1h);
      mma_tf32(qt, nxi0h, xr0h, nxi1h, xr1h, gi0h, gi1h);
      mma_tf32(qq, ngi0h, gr0h, ngi1h, gr1h, xi0h, xi1h);
      uint32_t h[4], l[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) split_tf32(qt[k], h[k], l[k]);
      xf[(nt * 2 + 0) * 32 + L.lane] = make_float4(__uint_as_float(h[0]), __uint_as_float(h[1]),
                                                   __uint_as_float(h[2]), __uint_as_float(h[3]));
      xf[(nt * 2 + 1) * 32 + L.lane] = make_float4(__uint_as_float(l[0]), __uint_as_float(l[1]),
                                                   __uint_as_float(l[2]), __uint_as_float(l[3]));
#pragma unroll
      for (int k = 0; k < 4; ++k) w[nt][k] = tg * qq[k];
    }
  }

  // Per-instance setup from the raw channel in c.Hs (and the targets in c.tks):
  // W^(0) into w, the update's B fragments into xf, H's hi / lo parts (PRE, in
  // place of the raw channel and into hlo); with xraw, also the raw conj(H) B
  // fragments of the update layout, (Re X[2q][8nt+g], Re X[2q+1][8nt+g],
  // Im X[2q][8nt+g], Im X[2q+1][8nt+g]) at [nt][lane].  Returns the instance
  // flags; invL: the paper layer's step normalisation.
  // With BASIS, FP64-path instances of the projected layer run in an orthonormal
  // basis of the channel's row space (Base::fp64_basis: U over the raw channel,
  // X = conj(U), S~^T at OFF_ST, *basis_out set); else their Q is formed in FP64.
  template <bool BASIS = false>
  __device__ static int setup(Ctx& c, const Lane& L, const SolveArgs& A, float4* xf, float4* hlo,
                              WT& w, float& invL, float4* xraw, bool* basis_out = nullptr) {
    bool basis = false;
    float2* const St = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(c.Qs) - OFF_Q + OFF_ST);
    float e[4];
    // ---- setup: lane's own conj(H) entries (user g, antennas 8s + 2q + h)
    int fl = 0;
    invL = 1.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float4 hv = *reinterpret_cast<const float4*>(c.Hs + L.g * MB + 8 * s + 2 * L.q);
      w[s][0] = hv.x;
      w[s][1] = hv.z;
      w[s][2] = -hv.y;
      w[s][3] = -hv.w;
    }
    bool fast = true;  // projected layer: FP32 register inverse and MMA-formed Q
    if constexpr (MODE == kModeProj) {
      residual<false>(L, c.Hs, nullptr, nullptr, w, c.tks, false, e);  // conj(H) H^T = G^T
      float gi[4];
      fast = gram_inverse(L, e, A.cond_thr, gi);
      if (fast) {
        // xf lies outside the raw channel, which the other lanes still read
        q_mma(L, c.Hs, gi, c.tks[L.g], xf, w);
      } else if constexpr (BASIS) {
        fl = Base::fp64_basis(c, St);  // U over the channel, conj(U) into Qs, S~^T
        basis = !(fl & PRECODE_F_SINGULAR);
      } else {
        fl = Base::fp64_inverse(c);  // G^{-1} in FP64 into the reduction buffer
        if (!(fl & PRECODE_F_SINGULAR)) {
          // Q = conj(G^{-1} H) in FP64, rounded once, into Qs (natural); one entry
          // at a time keeps this rare path light on registers
          const double2* Gi = reinterpret_cast<const double2*>(c.red);
#pragma unroll 1
          for (int idx = L.lane; idx < KB * MB; idx += 32) {
            const int k = idx / MB, m = idx - k * MB;
            double zr = 0.0, zi = 0.0;
#pragma unroll
            for (int l = 0; l < KB; ++l) {
              const double2 gkl = Gi[k * KB + l];
              const float2 x = c.Hs[l * MB + m];
              zr += gkl.x * x.x - gkl.y * x.y;
              zi += gkl.x * x.y + gkl.y * x.x;
            }
            c.Qs[idx] = make_float2((float)zr, (float)-zi);
          }
          __syncwarp();
        }
      }
    } else if (A.opts & OPT_STEP_NORMALISED) {
      residual<false>(L, c.Hs, nullptr, nullptr, w, c.tks, false, e);  // conj(H) H^T = G^T
      *reinterpret_cast<float4*>(c.Es + L.g * KB + 2 * L.q) = make_float4(e[0], e[2], e[1], e[3]);
      __syncwarp();
      invL = Base::inv_gershgorin(c);
    }
    const bool singular = (fl & PRECODE_F_SINGULAR) != 0;
    if (xraw) {  // raw conj(H) B fragments, read before the channel area is reused
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float2 h0 = c.Hs[(2 * L.q) * MB + 8 * nt + L.g];
        const float2 h1 = c.Hs[(2 * L.q + 1) * MB + 8 * nt + L.g];
        xraw[nt * 32 + L.lane] = make_float4(h0.x, h1.x, -h0.y, -h1.y);
      }
    }
    // ---- phase change: the layer buffers overwrite the setup buffers, so each
    // operand is read out (into registers) before its area is reused.
    {
      float4* const hh = reinterpret_cast<float4*>(c.Hs);
      // update fragments X[2q][8nt+g], X[2q+1][8nt+g], split into xf
      auto put_x = [&](int nt, float2 x0, float2 x1, float csign) {
        uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
        split_tf32(x0.x, h0, l0);
        split_tf32(x1.x, h1, l1);
        split_tf32(csign * x0.y, h2, l2);
        split_tf32(csign * x1.y, h3, l3);
        xf[(nt * 2 + 0) * 32 + L.lane] = make_float4(__uint_as_float(h0), __uint_as_float(h1),
                                                     __uint_as_float(h2), __uint_as_float(h3));
        xf[(nt * 2 + 1) * 32 + L.lane] = make_float4(__uint_as_float(l0), __uint_as_float(l1),
                                                     __uint_as_float(l2), __uint_as_float(l3));
      };
      // H hi parts in place of the raw channel, lo parts beside them, from the
      // lane's own entries v[s] = (Re, Re, Im, Im) at antennas 8s + 2q + {0, 1}
      auto put_h = [&](const float (&v)[8][4]) {
#pragma unroll
        for (int s = 0; s < 8; ++s) {
          uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
          split_tf32(v[s][0], h0, l0);
          split_tf32(v[s][1], h1, l1);
          split_tf32(v[s][2], h2, l2);
          split_tf32(v[s][3], h3, l3);
          hh[s * 32 + L.lane] = make_float4(__uint_as_float(h0), __uint_as_float(h1),
                                            __uint_as_float(h2), __uint_as_float(h3));
          hlo[s * 32 + L.lane] = make_float4(__uint_as_float(l0), __uint_as_float(l1),
                                             __uint_as_float(l2), __uint_as_float(l3));
        }
      };
      if constexpr (MODE == kModePGD) {
        // X = conj(H) from the raw channel; xf lies outside it
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
          put_x(nt, c.Hs[(2 * L.q) * MB + 8 * nt + L.g], c.Hs[(2 * L.q + 1) * MB + 8 * nt + L.g], -1.f);
        if constexpr (PRE) {
          __syncwarp();
          float v[8][4];  // w = conj(H) = W^(0) stays live
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            v[s][0] = w[s][0];
            v[s][1] = w[s][1];
            v[s][2] = -w[s][2];
            v[s][3] = -w[s][3];
          }
          put_h(v);
        }
      } else {
        // H re-read from the raw channel (w is rebuilt from Q below); all lanes
        // read before any overwrites it
        if constexpr (PRE) {
          float v[8][4];
#pragma unroll
          for (int s = 0; s < 8; ++s) {
            const float4 hv = *reinterpret_cast<const float4*>(c.Hs + L.g * MB + 8 * s + 2 * L.q);
            v[s][0] = hv.x;
            v[s][1] = hv.z;
            v[s][2] = hv.y;
            v[s][3] = hv.w;
          }
          __syncwarp();
          put_h(v);
        }
        if (!fast) {
          // X = Q from the FP64 path: tiles 4..7 of xf lie in the Gauss-Jordan
          // area, tiles 0..3 over Q
          const float2 z = make_float2(0.f, 0.f);
#pragma unroll
          for (int nt = 4; nt < 8; ++nt)
            put_x(nt, singular ? z : c.Qs[(2 * L.q) * MB + 8 * nt + L.g],
                  singular ? z : c.Qs[(2 * L.q + 1) * MB + 8 * nt + L.g], 1.f);
          if (basis) {  // W^(0) = S~^T conj(U) (the ZF precoder), row g; Qs = conj(U)
#pragma unroll
            for (int s = 0; s < 8; ++s)
#pragma unroll
              for (int k = 0; k < 4; ++k) w[s][k] = 0.f;
#pragma unroll 1
            for (int j = 0; j < KB; ++j) {
              const float2 sj = St[L.g * KB + j];
#pragma unroll
              for (int s = 0; s < 8; ++s) {
                const float4 qv = *reinterpret_cast<const float4*>(c.Qs + j * MB + 8 * s + 2 * L.q);
                w[s][0] += sj.x * qv.x - sj.y * qv.y;
                w[s][1] += sj.x * qv.z - sj.y * qv.w;
                w[s][2] += sj.x * qv.y + sj.y * qv.x;
                w[s][3] += sj.x * qv.w + sj.y * qv.z;
              }
            }
          } else {
            const float tg = c.tks[L.g];  // W^(0) = S Q
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
          float2 x0[4], x1[4];
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) {
            x0[nt] = singular ? z : c.Qs[(2 * L.q) * MB + 8 * nt + L.g];
            x1[nt] = singular ? z : c.Qs[(2 * L.q + 1) * MB + 8 * nt + L.g];
          }
          __syncwarp();
#pragma unroll
          for (int nt = 0; nt < 4; ++nt) put_x(nt, x0[nt], x1[nt], 1.f);
        }
      }
    }
    __syncwarp();
    if (basis_out) *basis_out = basis;
    return fl;
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
    c.Qs = reinterpret_cast<float2*>(gs + OFF_Q);
    c.red = reinterpret_cast<float*>(gs + OFF_RED);
    c.Es = reinterpret_cast<float2*>(gs + OFF_E);
    c.nrm = nullptr;
    c.tks = reinterpret_cast<float*>(gs + OFF_SC);
    c.dsc = c.tks + KB;
    c.piv = c.dsc + KB;
    c.misc = reinterpret_cast<int*>(c.piv + KB);
    c.wsum = reinterpret_cast<float*>(c.misc + 8);
    c.bar = reinterpret_cast<uint64_t*>(gs + OFF_BAR);
    float4* const xf = reinterpret_cast<float4*>(gs + OFF_XF);
    float4* const hlo = reinterpret_cast<float4*>(gs + OFF_LO);
    float* const nb = reinterpret_cast<float*>(gs + OFF_NB);
    float* const fb = reinterpret_cast<float*>(gs + OFF_FB);
    if (c.g == 0)
      for (int q = 0; q < NHB; ++q) mbar_init(c.bar + q, 1);
    fence_mbar_init();
    __syncthreads();

    auto hbuf = [&](int qb) { return reinterpret_cast<float2*>(gs + (qb == 0 ? 0 : OFF_H1)); };
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
      if (c.g != 0 || it >= n_inst || (A.opts & OPT_STALL_COPY)) return;
      int64_t inst, h_off, w_off, t_off;
      locate(it, inst, h_off, w_off, t_off);
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(c.bar + qb, KB * MB * 8);
      bulk_g2s(hbuf(qb), A.H + h_off, KB * MB * 8, c.bar + qb);
    };
    const int64_t first = (int64_t)blockIdx.x * C::GROUPS + c.gid;
    for (int qb = 0; qb < NHB; ++qb) issue_copy(first + qb * stride, qb);
    int cur = 0;
    WT w;
    float e[4];
#pragma unroll 1
    for (int64_t it = first; it < n_inst; it += stride, cur = (cur + 1) % NHB) {
      int64_t inst, h_off, w_off, t_off;
      locate(it, inst, h_off, w_off, t_off);
      c.K = KB;
      c.M = MB;
      c.Hs = hbuf(cur);
      const float4* const hhi = reinterpret_cast<const float4*>(c.Hs);
      const uint32_t par = (phases >> cur) & 1u;
      __syncwarp();
      if (c.g < KB) c.tks[c.g] = A.t[t_off + c.g];
      if (c.g == 0) c.misc[0] = mbar_wait_bounded(c.bar + cur, par, copy_wait_ns(A)) ? 1 : 0;
      __syncwarp();
      if (c.misc[0] == 0) {
        if (c.g == 0) {
          atomicAdd(A.err, 1ull);
          if (A.flags) A.flags[inst] = PRECODE_F_TIMEOUT;
          c.misc[1] = mbar_wait_bounded(c.bar + cur, par, copy_wait_ns(A)) ? 1 : 0;
        }
        __syncwarp();
        if (c.misc[1] == 0) return;
        phases ^= 1u << cur;
        issue_copy(it + NHB * stride, cur);
        continue;
      }
      if (c.g != 0) mbar_wait_bounded(c.bar + cur, par, copy_wait_ns(A));
      phases ^= 1u << cur;

      float invL;
      bool basis = false;  // FP64 path: the layers run in an orthonormal basis
      const int fl0 = setup<MODE == kModeProj>(c, L, A, xf, hlo, w, invL, nullptr, &basis);
      int fl = fl0;
      const bool singular = (fl & PRECODE_F_SINGULAR) != 0;

      // ---- layers
      const int T = A.T;
      float rs = 0.f;
      if (!singular) {
#pragma unroll 1
        for (int l = 0; l < T; ++l) {
          if constexpr (MODE == kModeProj) {
            shrink(L, fb, colsum(L, nb, w), fmaxf(__ldg(A.step + l), 0.f), w);
            residual<PRE>(L, c.Hs, hhi, hlo, w, c.tks, !basis, e);
            if (basis) {  // S~^T[g][2q], S~^T[g][2q + 1]
              const float4 v = *reinterpret_cast<const float4*>(
                  reinterpret_cast<const float2*>(reinterpret_cast<const unsigned char*>(c.tks) - OFF_SC + OFF_ST) + L.g * KB + 2 * L.q);
              e[0] -= v.x;
              e[1] -= v.z;
              e[2] -= v.y;
              e[3] -= v.w;
            }
            update(L, xf, e, w);
          } else {
            const float eta = __ldg(A.step + l) * invL;
            residual<PRE>(L, c.Hs, hhi, hlo, w, c.tks, true, e);
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] *= eta;
            update(L, xf, e, w);
            shrink(L, fb, colsum(L, nb, w), fmaxf(fmaxf(__ldg(A.lam + l), 0.f) * eta, 0.f), w);
          }
        }
        if (A.resid) {
          if (basis) {  // against the channel itself, from global memory
            int64_t i0, ho, wo, to;
            locate(it, i0, ho, wo, to);
            __syncwarp();  // every lane is done with U's fragments
#pragma unroll 1
            for (int s = 0; s < 8; ++s) {
              const float4 v = *reinterpret_cast<const float4*>(A.H + ho + L.g * MB + 8 * s + 2 * L.q);
              if constexpr (PRE) {  // hi / lo fragments (Hr0, Hr1, Hi0, Hi1)
                uint32_t h0, l0, h1, l1, h2, l2, h3, l3;
                split_tf32(v.x, h0, l0);
                split_tf32(v.z, h1, l1);
                split_tf32(v.y, h2, l2);
                split_tf32(v.w, h3, l3);
                const_cast<float4*>(hhi)[s * 32 + L.lane] =
                    make_float4(__uint_as_float(h0), __uint_as_float(h1), __uint_as_float(h2), __uint_as_float(h3));
                hlo[s * 32 + L.lane] =
                    make_float4(__uint_as_float(l0), __uint_as_float(l1), __uint_as_float(l2), __uint_as_float(l3));
              } else {
                *reinterpret_cast<float4*>(c.Hs + L.g * MB + 8 * s + 2 * L.q) = v;
              }
            }
            __syncwarp();
          }
          residual<PRE>(L, c.Hs, hhi, hlo, w, c.tks, true, e);
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
      const float2 r2 = colsum(L, nb, w);
      float o = sqrtf(r2.x) + sqrtf(r2.y);
#pragma unroll
      for (int msk = 1; msk < 32; msk <<= 1) o += __shfl_xor_sync(0xffffffffu, o, msk);
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
      __syncwarp();  // norm partials read out before the next instance
    }
  }
};

template <int MODE, int NW, int MINB, bool DB>
__global__ void __launch_bounds__(NW * 32, MINB) solve_tc_kernel(SolveArgs A) {
  SolveTC<MODE, NW, DB>::run(A);
}

}  // namespace precode
