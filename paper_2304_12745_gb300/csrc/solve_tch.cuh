// Solve kernel for K = 8 users, M = 64 antennas (projected layer; the paper layer
// with MODE = kModePGD) with every contraction as split-FP16 warp MMAs (m16n8k16):
// one warp per instance, the same lane ownership as the TF32 kernel (lane (g, q)
// holds user g's W at antennas 8s + 2q + {0, 1}), half the MMAs of the TF32 split
// for the same accuracy, and half its fragment traffic through shared memory.
//
// FP16 covers a narrow exponent range, so every instance is solved in scaled
// units made of exact powers of two, under which the projected iteration is
// equivariant: with D = diag(d_k) and a scalar b,
//   H' = D H,  t'_k = b d_k t_k,  W' = b W,  mu' = b mu,  X = Q' = G'^{-T} H'^* = D^{-1} Q,
// every iterate is W' = b W and the residual is E' = b E D.  d_k puts the largest
// component of user k's channel row in [1/2, 1), so every row of H' and of Q' is
// of order one whatever the spread of the users' gains (a weak user's row would
// otherwise fall into FP16's subnormals, and its errors are amplified by 1 / |h_k|
// in W); b puts max(|W^(0)'|, t') in [2^6, 2^7).  An instance whose Q' exceeds
// 2^13 (an equilibrated Gram condition far beyond FP32 accuracy, FP64 path only)
// is reported as singular.  W, the objective and the residual are scaled back on
// the way out.
//
// Per layer, reduction over antennas (residual E = W H^T, 16 antennas per MMA):
//   A = (Re W, Im W) rows, B = Re H or Im H, accumulators ar / ai,
//   E_re = [ar]_g - [ai]_g+8,  E_im = [ai]_g + [ar]_g+8;
// reduction over users (update W -= E X, k = (Re, Im) x 8 users per MMA):
//   A rows g: (-E_re, +E_im), rows g+8: (-E_im, -E_re), B = (Re X; Im X).
// Once per instance: the Gram matrix G'^T as a residual with W = conj(H') on the
// same H' fragments, its Gauss-Jordan inverse in registers as in the TF32 kernel
// (FP64 path for ill-conditioned instances), then Q' and Q'^T by split-FP16 MMAs
// (q_tile_h).
#pragma once

#include "f16mma.cuh"
#include "solve_tc.cuh"

namespace precode {

// HOSTIO: the channel is read with plain 16-byte loads (no bulk async copy),
// so H, W, t and the outputs may live in page-locked host memory mapped into the
// device's address space (zero-copy over the host link).
//
// MODE = kModePGD (the paper layer) uses one global power of two on H instead of
// the per-user scales (its iteration is equivariant under global scaling only):
// H' = a H, W' = (b / a) W, t' = b t, eta' = eta / a^2, tau' = (b / a) tau, so
// W^(0)' = (b / a^2) conj(H'), X = conj(H') and E' = b E.  A weak user's channel
// row may then sit in FP16's subnormals; the rounding that costs is absolute and
// small against the instance's norms (that user's W row stays of the order of its
// channel row in this iteration).
template <int NW, bool HOSTIO = false, int MODE = kModeProj>
struct SolveTCH : SolveTC<MODE, NW, false> {
  using S = SolveTC<MODE, NW, false>;
  using Base = typename S::Base;
  using C = typename S::C;
  using Ctx = typename S::Ctx;
  using Lane = typename S::Lane;
  using WT = typename S::WT;
  static constexpr int KB = 8, MB = 64;
  // antenna tiles per update batch (4 independent MMA chains; 2 keeps the paper
  // layer's build inside its 128 registers)
  static constexpr int UG = MODE == kModeProj ? 4 : 2;
  // Per-warp shared memory, two overlaid phases (bytes):
  //   setup : H (raw channel, scaled in place) | H' hi / lo FP16 fragments (written
  //           first, for the Gram and the layers; FP64 scratch and Q on the FP64
  //           path, which writes the fragments again) | G^{-1} (FP64) | Gram
  //   layers: X fragments (over the raw channel) | H' hi / lo fragments | norm
  //           partials | factors
  //   both  : t, scalars, copy barrier
  static constexpr int H_BYTES = KB * MB * 8;
  static constexpr int OFF_Q = H_BYTES;                   // setup (FP64 path), 4 KB
  static constexpr int OFF_RED = OFF_Q + KB * MB * 8;     // setup, 1 KB
  static constexpr int OFF_E = OFF_RED + KB * KB * 16;    // setup, 512 B
  static constexpr int OFF_XF = 0;                        // layers, 4 KB
  static constexpr int OFF_HH = H_BYTES;                  // setup and layers: hi fragments
  static constexpr int OFF_HL = H_BYTES + H_BYTES / 2;    //   and lo fragments
  static constexpr int OFF_NB = 2 * H_BYTES;              // layers, 2 KB
  static constexpr int OFF_FB = OFF_NB + 2048;            // layers, 256 B
  static constexpr int OFF_ST = OFF_FB + 256;             // S~^T of the FP64 path, 512 B
  static constexpr int OFF_SC = (OFF_ST + 512 > OFF_E + KB * KB * 8) ? OFF_ST + 512 : OFF_E + KB * KB * 8;
  static constexpr int OFF_BAR = OFF_SC + C::SC_BYTES;
  static constexpr int GROUP_STRIDE = align_up(OFF_BAR + 8, 16);
  static constexpr int SMEM_BYTES = NW * GROUP_STRIDE;
  static constexpr float QMAX = 8192.f;  // bound on |Q'| entries

  // E = W H^T from the FP16 H fragments (hh / hl: [pair][lane] of (Hr block 2p,
  // Hr block 2p+1, Hi block 2p, Hi block 2p+1) pairs); two pairs of blocks at a
  // time, term by term (lo terms first).
  __device__ __forceinline__ static void residual_h(const Lane& L, const uint4* hh, const uint4* hl,
                                                    const WT& w, float (&e)[4]) {
    float ar[2][4], ai[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) ar[i][k] = ai[i][k] = 0.f;
#pragma unroll
    for (int p0 = 0; p0 < 4; p0 += 2) {
      uint4 bh[2], bl[2];
      uint32_t ah[2][4], al[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const int p = p0 + u;
        bh[u] = hh[p * 32 + L.lane];
        bl[u] = hl[p * 32 + L.lane];
        split_h2(w[2 * p][0], w[2 * p][1], ah[u][0], al[u][0]);          // Re W, block 2p
        split_h2(w[2 * p][2], w[2 * p][3], ah[u][1], al[u][1]);          // Im W, block 2p
        split_h2(w[2 * p + 1][0], w[2 * p + 1][1], ah[u][2], al[u][2]);  // Re W, block 2p+1
        split_h2(w[2 * p + 1][2], w[2 * p + 1][3], ah[u][3], al[u][3]);  // Im W, block 2p+1
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mma_f16(ar[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bl[u].x, bl[u].y);
        mma_f16(ai[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bl[u].z, bl[u].w);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mma_f16(ar[u], al[u][0], al[u][1], al[u][2], al[u][3], bh[u].x, bh[u].y);
        mma_f16(ai[u], al[u][0], al[u][1], al[u][2], al[u][3], bh[u].z, bh[u].w);
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        mma_f16(ar[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bh[u].x, bh[u].y);
        mma_f16(ai[u], ah[u][0], ah[u][1], ah[u][2], ah[u][3], bh[u].z, bh[u].w);
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
  }

  // W -= E X with the FP16 X fragments (xf: [tile][lane] of (Re X hi, Im X hi,
  // Re X lo, Im X lo) pairs over users 2q, 2q+1 at antenna 8nt + g).  The tensor
  // cores' FP32 accumulation does not round to nearest: adding each update to W
  // inside the MMA shrinks W's magnitude by about half an ulp per layer, a drift
  // that grows linearly with the number of layers (1.5e-4 relative after the
  // classical PGD's 5,000 layers).  The paper layer, which runs thousands of
  // layers as the classical PGD, therefore accumulates the product from zero and
  // adds it to W with a rounded FP32 add.  The projected layer (tens of layers)
  // keeps the MMA's own accumulation into W (the extra adds and accumulators cost
  // 6 % of its time): its drift is below T 2^-24 relative.
  __device__ __forceinline__ static void update_h(const Lane& L, const uint4* xf, const float (&e)[4],
                                                  WT& w) {
    uint32_t h01, l01, h23, l23;
    split_h2(e[0], e[1], h01, l01);
    split_h2(e[2], e[3], h23, l23);
    const uint32_t nh01 = neg_h2(h01), nl01 = neg_h2(l01), nh23 = neg_h2(h23), nl23 = neg_h2(l23);
#pragma unroll
    for (int nt0 = 0; nt0 < 8; nt0 += UG) {
      uint4 x[UG];
      float d[UG][4];
#pragma unroll
      for (int u = 0; u < UG; ++u) {
        x[u] = xf[(nt0 + u) * 32 + L.lane];
#pragma unroll
        for (int k = 0; k < 4; ++k) d[u][k] = 0.f;
      }
      if constexpr (MODE == kModeProj) {  // into W directly (see above)
#pragma unroll
        for (int u = 0; u < UG; ++u) mma_f16(w[nt0 + u], nh01, nh23, h23, nh01, x[u].z, x[u].w);
#pragma unroll
        for (int u = 0; u < UG; ++u) mma_f16(w[nt0 + u], nl01, nl23, l23, nl01, x[u].x, x[u].y);
#pragma unroll
        for (int u = 0; u < UG; ++u) mma_f16(w[nt0 + u], nh01, nh23, h23, nh01, x[u].x, x[u].y);
      } else {
#pragma unroll
        for (int u = 0; u < UG; ++u) mma_f16(d[u], nh01, nh23, h23, nh01, x[u].z, x[u].w);
#pragma unroll
        for (int u = 0; u < UG; ++u) mma_f16(d[u], nl01, nl23, l23, nl01, x[u].x, x[u].y);
#pragma unroll
        for (int u = 0; u < UG; ++u) mma_f16(d[u], nh01, nh23, h23, nh01, x[u].x, x[u].y);
#pragma unroll
        for (int u = 0; u < UG; ++u)
#pragma unroll
          for (int k = 0; k < 4; ++k) w[nt0 + u][k] += d[u][k];
      }
    }
  }

  // Q' tile nt into wq (W's layout, rows user g, antennas 8nt + 2q + {0, 1}) and
  // Q'^T tile nt into qt (the update's X values (Re Q'[2q][8nt+g], Re Q'[2q+1][8nt+g],
  // Im Q'[2q][8nt+g], Im Q'[2q+1][8nt+g])), as split-FP16 MMAs from the lane's
  // G'^{-T} entries (g01 = Re, g23 = Im, hi / lo, scaled into FP16's range) and the
  // scaled channel.  Both products reduce over the users; the channel pair
  // conj(H'[2q][8nt+g]), conj(H'[2q+1][8nt+g]) is the B operand of the first and the
  // A operand of the second, the G'^{-T} pair the other way round:
  //   Q'   = G'^{-T} X:   A = (Re G, Im G, -Im G, Re G) rows,  B = (Re X; Im X);
  //   Q'^T = X^T G'^{-1}: A = (Re X, Im X, -Im X, Re X) rows,  B = (Re G; Im G).
  __device__ __forceinline__ static void q_tile_h(const Lane& L, const float2* Hs, uint32_t gh01,
                                                  uint32_t gl01, uint32_t gh23, uint32_t gl23,
                                                  int nt, float (&qt)[4], float (&wq)[4]) {
    const float2 h0 = Hs[(2 * L.q) * MB + 8 * nt + L.g];
    const float2 h1 = Hs[(2 * L.q + 1) * MB + 8 * nt + L.g];
    uint32_t xrh, xrl, xih, xil;  // X = conj(H')
    split_h2(h0.x, h1.x, xrh, xrl);
    split_h2(-h0.y, -h1.y, xih, xil);
    const uint32_t ngh23 = neg_h2(gh23), ngl23 = neg_h2(gl23);
    const uint32_t nxih = neg_h2(xih), nxil = neg_h2(xil);
#pragma unroll
    for (int k = 0; k < 4; ++k) qt[k] = wq[k] = 0.f;
    mma_f16(wq, gh01, gh23, ngh23, gh01, xrl, xil);
    mma_f16(qt, xrh, xih, nxih, xrh, gl01, gl23);
    mma_f16(wq, gl01, gl23, ngl23, gl01, xrh, xih);
    mma_f16(qt, xrl, xil, nxil, xrl, gh01, gh23);
    mma_f16(wq, gh01, gh23, ngh23, gh01, xrh, xih);
    mma_f16(qt, xrh, xih, nxih, xrh, gh01, gh23);
  }

  // H' hi / lo B fragments of the residual from the lane's own channel entries hv[s]
  // (H'[g][8s+2q], H'[g][8s+2q+1]): [pair p][lane] of (Re block 2p, Re block 2p+1,
  // Im block 2p, Im block 2p+1).
  __device__ __forceinline__ static void put_h_fragments(const Lane& L, const float4 (&hv)[8],
                                                         uint4* hh, uint4* hl) {
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const float4 a = hv[2 * p], b = hv[2 * p + 1];
      uint32_t rah, ral, rbh, rbl, iah, ial, ibh, ibl;
      split_h2(a.x, a.z, rah, ral);  // Re H', block 2p
      split_h2(b.x, b.z, rbh, rbl);  // Re H', block 2p+1
      split_h2(a.y, a.w, iah, ial);  // Im H', block 2p
      split_h2(b.y, b.w, ibh, ibl);  // Im H', block 2p+1
      hh[p * 32 + L.lane] = make_uint4(rah, rbh, iah, ibh);
      hl[p * 32 + L.lane] = make_uint4(ral, rbl, ial, ibl);
    }
  }

  __device__ __forceinline__ static float warp_max(float v) {
#pragma unroll
    for (int msk = 1; msk < 32; msk <<= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, msk));
    return v;
  }
  // 2^-e with v = f 2^e, f in [1/2, 1); 1 for zero or non-finite v
  __device__ __forceinline__ static float inv_pow2_of(float v) {
    if (!(v > 0.f) || !(v <= FLT_MAX)) return 1.f;
    int ex;
    frexpf(v, &ex);
    return ldexpf(1.f, -ex);
  }

  // Per-instance setup: the scaled problem (d_k^{-1} into c.dsc, t' into c.tks),
  // the H' fragments (at OFF_HH / OFF_HL), the X fragments (into xf, over the raw
  // channel) and W^(0)' into w; b into beta.  With xraw, also the unscaled conj(H)
  // B fragments of the TF32 update layout, (Re X[2q][8nt+g], Re X[2q+1][8nt+g],
  // Im X[2q][8nt+g], Im X[2q+1][8nt+g]) at [nt][lane], taken before the scaling.
  // Returns the instance flags.
  // With BASIS, FP64-path instances run in an orthonormal basis of the channel's
  // row space (S~^T at OFF_ST, `basis` set); else their Q is formed in FP64.
  // fin: the instance's resident factor slot (its G'^{-T} replaces the Gram matrix
  // and its inversion when the slot holds the FP32 path's); fout: the slot that
  // receives them.
  template <bool BASIS = false>
  __device__ static int setup(Ctx& c, const Lane& L, const SolveArgs& A, uint4* xf, WT& w,
                              float& beta, float4* xraw = nullptr, bool* basis_out = nullptr,
                              const float2* fin = nullptr, float2* fout = nullptr) {
    float2* const Hs = c.Hs;
    uint4* const hh = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Hs) + OFF_HH);
    uint4* const hl = reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Hs) + OFF_HL);
    if (xraw) {
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float2 h0 = Hs[(2 * L.q) * MB + 8 * nt + L.g];
        const float2 h1 = Hs[(2 * L.q + 1) * MB + 8 * nt + L.g];
        xraw[nt * 32 + L.lane] = make_float4(h0.x, h1.x, -h0.y, -h1.y);
      }
      __syncwarp();  // read before any lane scales its row
    }
    // ---- per-user scales on the lane's own entries: row g of H' = d_g H[g] (in
    // place, for the transposed reads of Q), t'_g = d_g t_g; then the H' fragments
    // and W = conj(H') for the Gram
    int fl = 0;
    float e[4];
    {
      float4 hv[8];
      float hm = 0.f;
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        hv[s] = *reinterpret_cast<const float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
        hm = fmaxf(hm, fmaxf(fmaxf(fabsf(hv[s].x), fabsf(hv[s].y)),
                             fmaxf(fabsf(hv[s].z), fabsf(hv[s].w))));
      }
      hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, 1));  // the 4 lanes of row g
      hm = fmaxf(hm, __shfl_xor_sync(0xffffffffu, hm, 2));
      const float dg = inv_pow2_of(hm);
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        hv[s] = make_float4(dg * hv[s].x, dg * hv[s].y, dg * hv[s].z, dg * hv[s].w);
        *reinterpret_cast<float4*>(Hs + L.g * MB + 8 * s + 2 * L.q) = hv[s];
        w[s][0] = hv[s].x;
        w[s][1] = hv[s].z;
        w[s][2] = -hv[s].y;
        w[s][3] = -hv[s].w;
      }
      put_h_fragments(L, hv, hh, hl);
      if (L.q == 0) {
        c.tks[L.g] *= dg;
        c.dsc[L.g] = 1.f / dg;
      }
    }
    __syncwarp();

    // ---- Gram G'^T (split FP16, as a layer's residual with W = conj(H')), inverse, Q
    float gi[4];
    bool fast;
    if (fin && fin[KB * KB].x == 1.f) {  // resident: G'^{-T}[g][2q + h] of this channel
      const float2 f0 = fin[L.g * KB + 2 * L.q], f1 = fin[L.g * KB + 2 * L.q + 1];
      gi[0] = f0.x;
      gi[1] = f1.x;
      gi[2] = f0.y;
      gi[3] = f1.y;
      fast = true;
    } else {
      residual_h(L, hh, hl, w, e);
      fast = S::gram_inverse(L, e, A.cond_thr, gi);
    }
    if (fout) {
      fout[L.g * KB + 2 * L.q] = make_float2(gi[0], gi[2]);
      fout[L.g * KB + 2 * L.q + 1] = make_float2(gi[1], gi[3]);
      if (L.lane == 0) fout[KB * KB] = make_float2(fast ? 1.f : 0.f, 0.f);
    }
    float qt[8][4];
    bool singular = false, basis = false;
    if (fast) {
      // G'^{-T} into FP16's range by a power of two (undone on the products)
      float gm = 0.f;
#pragma unroll
      for (int k = 0; k < 4; ++k) gm = fmaxf(gm, fabsf(gi[k]));
      const float gsc = inv_pow2_of(warp_max(gm)), igs = 1.f / gsc;
      uint32_t gh01, gl01, gh23, gl23;
      split_h2(gsc * gi[0], gsc * gi[1], gh01, gl01);
      split_h2(gsc * gi[2], gsc * gi[3], gh23, gl23);
      const float tg = c.tks[L.g] * igs;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        float wq[4];
        q_tile_h(L, Hs, gh01, gl01, gh23, gl23, nt, qt[nt], wq);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          qt[nt][k] *= igs;
          w[nt][k] = tg * wq[k];
        }
      }
    } else if constexpr (BASIS) {
      // FP64 path in an orthonormal basis of the scaled channel's row space: U
      // replaces H' (rows of unit norm, inside FP16's range), X = conj(U) and the
      // layers subtract S~^T (Base::fp64_basis; its scratch overlays the H'
      // fragments, which are written again from U)
      float2* const St = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(Hs) + OFF_ST);
      fl = Base::fp64_basis(c, St);
      singular = (fl & PRECODE_F_SINGULAR) != 0;
      basis = !singular;
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float2 x0 = singular ? make_float2(0.f, 0.f) : Hs[(2 * L.q) * MB + 8 * nt + L.g];
        const float2 x1 = singular ? make_float2(0.f, 0.f) : Hs[(2 * L.q + 1) * MB + 8 * nt + L.g];
        qt[nt][0] = x0.x;
        qt[nt][1] = x1.x;
        qt[nt][2] = -x0.y;
        qt[nt][3] = -x1.y;
#pragma unroll
        for (int k = 0; k < 4; ++k) w[nt][k] = 0.f;
      }
      if (!singular) {  // W^(0) = S~^T conj(U) (the ZF precoder), row g
#pragma unroll 1
        for (int j = 0; j < KB; ++j) {
          const float2 sj = St[L.g * KB + j];
#pragma unroll
          for (int nt = 0; nt < 8; ++nt) {
            const float4 u = *reinterpret_cast<const float4*>(Hs + j * MB + 8 * nt + 2 * L.q);
            // += sj * conj(u)
            w[nt][0] += sj.x * u.x + sj.y * u.y;
            w[nt][1] += sj.x * u.z + sj.y * u.w;
            w[nt][2] += sj.y * u.x - sj.x * u.y;
            w[nt][3] += sj.y * u.z - sj.x * u.w;
          }
        }
      }
      __syncwarp();  // U read out: the fragments from it
      float4 hv[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) hv[s] = *reinterpret_cast<const float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
      put_h_fragments(L, hv, hh, hl);
    } else {
      fl = Base::fp64_inverse(c);  // its scratch overlays the H' fragments
      singular = (fl & PRECODE_F_SINGULAR) != 0;
      if (!singular) {
        const double2* Gi = reinterpret_cast<const double2*>(c.red);
#pragma unroll 1
        for (int idx = L.lane; idx < KB * MB; idx += 32) {
          const int k = idx / MB, m = idx - k * MB;
          double zr = 0.0, zi = 0.0;
#pragma unroll
          for (int l = 0; l < KB; ++l) {
            const double2 gkl = Gi[k * KB + l];
            const float2 x = Hs[l * MB + m];
            zr += gkl.x * x.x - gkl.y * x.y;
            zi += gkl.x * x.y + gkl.y * x.x;
          }
          c.Qs[idx] = make_float2((float)zr, (float)-zi);
        }
        __syncwarp();
      }
      const float tg = c.tks[L.g];
#pragma unroll
      for (int nt = 0; nt < 8; ++nt) {
        const float2 x0 = singular ? make_float2(0.f, 0.f) : c.Qs[(2 * L.q) * MB + 8 * nt + L.g];
        const float2 x1 = singular ? make_float2(0.f, 0.f) : c.Qs[(2 * L.q + 1) * MB + 8 * nt + L.g];
        qt[nt][0] = x0.x;
        qt[nt][1] = x1.x;
        qt[nt][2] = x0.y;
        qt[nt][3] = x1.y;
        const float4 qv = singular ? make_float4(0.f, 0.f, 0.f, 0.f)
                                   : *reinterpret_cast<const float4*>(c.Qs + L.g * MB + 8 * nt + 2 * L.q);
        w[nt][0] = tg * qv.x;
        w[nt][1] = tg * qv.z;
        w[nt][2] = tg * qv.y;
        w[nt][3] = tg * qv.w;
      }
      __syncwarp();  // Q read out: the H' fragments again, from the scaled channel
      float4 hv[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) hv[s] = *reinterpret_cast<const float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
      put_h_fragments(L, hv, hh, hl);
    }
    // ---- range of Q', then the global scale b from W^(0)' and t'
    float qm = 0.f, wm = 0.f;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        qm = fmaxf(qm, fabsf(qt[nt][k]));
        wm = fmaxf(wm, fabsf(w[nt][k]));
      }
    qm = warp_max(qm);
    wm = warp_max(fmaxf(wm, fabsf(c.tks[L.lane & 7])));
    if (qm > QMAX && qm <= FLT_MAX) {  // beyond what FP16 fragments hold: reported as singular
      fl |= PRECODE_F_SINGULAR;
      singular = true;
    }
    beta = 128.f * inv_pow2_of(wm);
#pragma unroll
    for (int s = 0; s < 8; ++s)
#pragma unroll
      for (int k = 0; k < 4; ++k) w[s][k] = singular ? 0.f : beta * w[s][k];
    __syncwarp();  // every read of the raw channel, of Q and of t' done
    if (L.lane < KB) c.tks[L.lane] *= beta;
    if (basis) {  // S~^T in the same units as t'
      float2* const St = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(Hs) + OFF_ST);
      for (int idx = L.lane; idx < KB * KB; idx += 32) {
        const float2 v = St[idx];
        St[idx] = make_float2(beta * v.x, beta * v.y);
      }
    }
    if (basis_out) *basis_out = basis;
    // ---- X fragments over the raw channel
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
      uint32_t rh, rl, ih, il;
      split_h2(qt[nt][0], qt[nt][1], rh, rl);
      split_h2(qt[nt][2], qt[nt][3], ih, il);
      xf[nt * 32 + L.lane] = make_uint4(rh, ih, rl, il);
    }
    __syncwarp();
    return fl;
  }

  // Paper-layer setup: the scaled problem (t' into c.tks, d_k^{-1} = 1 into
  // c.dsc), X = conj(H') and the H' fragments, W^(0)' into w; the step factor
  // (eta' = step invLp), the threshold factor ba (tau' = ba lambda eta'), the output
  // factors f_out (W, objective) and f_res (residual).
  __device__ static void setup_pgd(Ctx& c, const Lane& L, const SolveArgs& A, uint4* xf, WT& w,
                                   float& invLp, float& ba, float& f_out, float& f_res) {
    float2* const Hs = c.Hs;
    float hm = 0.f;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const float4 hv = *reinterpret_cast<const float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
      hm = fmaxf(hm, fmaxf(fmaxf(fabsf(hv.x), fabsf(hv.y)), fmaxf(fabsf(hv.z), fabsf(hv.w))));
    }
    hm = warp_max(hm);
    const float alpha = inv_pow2_of(hm);
    const float tm = warp_max(fabsf(c.tks[L.lane & 7]));
    __syncwarp();
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      float4* p = reinterpret_cast<float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
      const float4 hv = *p;
      *p = make_float4(alpha * hv.x, alpha * hv.y, alpha * hv.z, alpha * hv.w);
    }
    __syncwarp();
    const float ia2 = 1.f / (alpha * alpha);
    invLp = ia2;
    if (A.opts & OPT_STEP_NORMALISED) {  // 1 / Gershgorin bound of G' = a^2 G
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        const float4 hv = *reinterpret_cast<const float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
        w[s][0] = hv.x;
        w[s][1] = hv.z;
        w[s][2] = -hv.y;
        w[s][3] = -hv.w;
      }
      float e[4];
      S::template residual<false>(L, Hs, nullptr, nullptr, w, c.tks, false, e);  // G'^T
      *reinterpret_cast<float4*>(c.Es + L.g * KB + 2 * L.q) = make_float4(e[0], e[2], e[1], e[3]);
      __syncwarp();
      invLp = Base::inv_gershgorin(c);
    }
    // W^(0)' = (b / a^2) conj(H') with max(|W^(0)'|, t') in [8, 16); the H'
    // fragments at OFF_HH / OFF_HL
    const float beta = 16.f * inv_pow2_of(fmaxf(alpha * hm * ia2, tm));
    const float c0 = beta * ia2;
    {
      float4 hv[8];
#pragma unroll
      for (int s = 0; s < 8; ++s) {
        hv[s] = *reinterpret_cast<const float4*>(Hs + L.g * MB + 8 * s + 2 * L.q);
        w[s][0] = c0 * hv[s].x;
        w[s][1] = c0 * hv[s].z;
        w[s][2] = -c0 * hv[s].y;
        w[s][3] = -c0 * hv[s].w;
      }
      put_h_fragments(L, hv,
                      reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Hs) + OFF_HH),
                      reinterpret_cast<uint4*>(reinterpret_cast<unsigned char*>(Hs) + OFF_HL));
    }
    uint4 xv[8];
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {  // X = conj(H') over users 2q, 2q + 1 at antenna 8nt + g
      const float2 h0 = Hs[(2 * L.q) * MB + 8 * nt + L.g];
      const float2 h1 = Hs[(2 * L.q + 1) * MB + 8 * nt + L.g];
      uint32_t rh, rl, ih, il;
      split_h2(h0.x, h1.x, rh, rl);
      split_h2(-h0.y, -h1.y, ih, il);
      xv[nt] = make_uint4(rh, ih, rl, il);
    }
    __syncwarp();  // every read of the channel (and of the Gershgorin scratch) done
    if (L.lane < KB) {
      c.tks[L.lane] *= beta;
      c.dsc[L.lane] = 1.f;
    }
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) xf[nt * 32 + L.lane] = xv[nt];  // over the raw channel
    __syncwarp();
    ba = beta * alpha;
    f_out = alpha / beta;
    f_res = 1.f / beta;
  }

  __device__ static void run(const SolveArgs& A) {
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
    uint4* const xf = reinterpret_cast<uint4*>(gs + OFF_XF);
    const uint4* const hh = reinterpret_cast<const uint4*>(gs + OFF_HH);
    const uint4* const hl = reinterpret_cast<const uint4*>(gs + OFF_HL);
    float* const nb = reinterpret_cast<float*>(gs + OFF_NB);
    float* const fb = reinterpret_cast<float*>(gs + OFF_FB);
    if (c.g == 0) mbar_init(c.bar, 1);
    fence_mbar_init();
    __syncthreads();

    uint32_t phase = 0;
    const int64_t n_inst = A.tbl ? (int64_t)(*A.count) : A.B;
    const int64_t stride = (int64_t)gridDim.x * NW;
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
    auto issue_copy = [&](int64_t it) {
      if (HOSTIO || c.g != 0 || it >= n_inst || (A.opts & OPT_STALL_COPY)) return;
      int64_t inst, h_off, w_off, t_off;
      locate(it, inst, h_off, w_off, t_off);
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(c.bar, KB * MB * 8);
      bulk_g2s(c.Hs, A.H + h_off, KB * MB * 8, c.bar);
    };
    const int64_t first = (int64_t)blockIdx.x * NW + c.gid;
    issue_copy(first);
    WT w;
    float e[4];
#pragma unroll 1
    for (int64_t it = first; it < n_inst; it += stride) {
      int64_t inst, h_off, w_off, t_off;
      locate(it, inst, h_off, w_off, t_off);
      __syncwarp();
      if (c.g < KB) c.tks[c.g] = A.t[t_off + c.g];
      if constexpr (HOSTIO) {  // the instance's channel, 16 bytes per lane and load
        const float4* src = reinterpret_cast<const float4*>(A.H + h_off);
        float4* dst = reinterpret_cast<float4*>(c.Hs);
        float4 v[KB * MB * 8 / 16 / 32];
#pragma unroll
        for (int j = 0; j < KB * MB * 8 / 16 / 32; ++j) v[j] = src[L.lane + 32 * j];
#pragma unroll
        for (int j = 0; j < KB * MB * 8 / 16 / 32; ++j) dst[L.lane + 32 * j] = v[j];
        __syncwarp();
      } else {
      if (c.g == 0) c.misc[0] = mbar_wait_bounded(c.bar, phase, copy_wait_ns(A)) ? 1 : 0;
      __syncwarp();
      if (c.misc[0] == 0) {
        if (c.g == 0) {
          atomicAdd(A.err, 1ull);
          if (A.flags) A.flags[inst] = PRECODE_F_TIMEOUT;
          c.misc[1] = mbar_wait_bounded(c.bar, phase, copy_wait_ns(A)) ? 1 : 0;
        }
        __syncwarp();
        if (c.misc[1] == 0) return;
        phase ^= 1u;
        issue_copy(it + stride);
        continue;
      }
      if (c.g != 0) mbar_wait_bounded(c.bar, phase, copy_wait_ns(A));
      phase ^= 1u;
      }

      float beta = 1.f, f_out, f_res, invLp = 1.f, ba = 1.f;
      int fl = 0;
      bool basis = false;  // FP64 path: the layers run in an orthonormal basis
      if constexpr (MODE == kModeProj) {
        const float2* fin = nullptr;
        float2* fout = nullptr;
        if (A.fac) {
          if (A.opts & OPT_FAC_EXPORT)
            fout = A.fac + inst * (int64_t)fac_stride(KB);
          else if (A.fidx && A.fidx[inst] >= 0)
            fin = A.fac + A.fidx[inst];
        }
        fl = setup<true>(c, L, A, xf, w, beta, nullptr, &basis, fin, fout);
        f_out = f_res = 1.f / beta;
      } else {
        setup_pgd(c, L, A, xf, w, invLp, ba, f_out, f_res);
      }
      const bool singular = (fl & PRECODE_F_SINGULAR) != 0;

      // ---- layers (scaled units)
      const int T = A.T;
      float rs = 0.f;
      if (!singular) {
#pragma unroll 1
        for (int l = 0; l < T; ++l) {
          if constexpr (MODE == kModeProj) {
            S::shrink(L, fb, S::colsum(L, nb, w), fmaxf(__ldg(A.step + l), 0.f) * beta, w);
            residual_h(L, hh, hl, w, e);
            if (basis) {  // S~^T[g][2q], S~^T[g][2q + 1]
              const float4 v = *reinterpret_cast<const float4*>(
                  reinterpret_cast<const float2*>(smem + c.gid * GROUP_STRIDE + OFF_ST) + L.g * KB + 2 * L.q);
              e[0] -= v.x;
              e[1] -= v.z;
              e[2] -= v.y;
              e[3] -= v.w;
            } else {
              if (2 * L.q == L.g) e[0] -= c.tks[L.g];
              if (2 * L.q + 1 == L.g) e[1] -= c.tks[L.g];
            }
            update_h(L, xf, e, w);
          } else {  // residual, gradient step, shrink (the paper's order)
            const float eta = __ldg(A.step + l) * invLp;
            residual_h(L, hh, hl, w, e);
            if (2 * L.q == L.g) e[0] -= c.tks[L.g];
            if (2 * L.q + 1 == L.g) e[1] -= c.tks[L.g];
#pragma unroll
            for (int k = 0; k < 4; ++k) e[k] *= eta;
            update_h(L, xf, e, w);
            S::shrink(L, fb, S::colsum(L, nb, w), fmaxf(fmaxf(__ldg(A.lam + l), 0.f) * eta, 0.f) * ba, w);
          }
        }
        if (A.resid) {
          if (basis) {  // against the channel itself: its H' fragments from global memory
            const float dg = 1.f / c.dsc[L.g];  // a power of two: exact
            float4 hv[8];
#pragma unroll
            for (int s = 0; s < 8; ++s) {
              const float4 v = *reinterpret_cast<const float4*>(A.H + h_off + L.g * MB + 8 * s + 2 * L.q);
              hv[s] = make_float4(dg * v.x, dg * v.y, dg * v.z, dg * v.w);
            }
            __syncwarp();
            put_h_fragments(L, hv, const_cast<uint4*>(hh), const_cast<uint4*>(hl));
            __syncwarp();
          }
          residual_h(L, hh, hl, w, e);
          if (2 * L.q == L.g) e[0] -= c.tks[L.g];
          if (2 * L.q + 1 == L.g) e[1] -= c.tks[L.g];
          // E' = b E D: columns 2q, 2q + 1 back to E (up to the 1 / b applied below)
          const float d0 = c.dsc[2 * L.q], d1 = c.dsc[2 * L.q + 1];
          rs = d0 * d0 * (e[0] * e[0] + e[2] * e[2]) + d1 * d1 * (e[1] * e[1] + e[3] * e[3]);
#pragma unroll
          for (int msk = 1; msk < 32; msk <<= 1) rs += __shfl_xor_sync(0xffffffffu, rs, msk);
        }
      } else {
        for (int k = 0; k < KB; ++k) rs += (c.tks[k] * c.dsc[k]) * (c.tks[k] * c.dsc[k]);
      }

      // ---- channel buffer free: next copy, then objective and W (original units)
      __syncwarp();
      issue_copy(it + stride);
      const float2 r2 = S::colsum(L, nb, w);
      float o = sqrtf(r2.x) + sqrtf(r2.y);
#pragma unroll
      for (int msk = 1; msk < 32; msk <<= 1) o += __shfl_xor_sync(0xffffffffu, o, msk);
#pragma unroll
      for (int s = 0; s < 8; ++s)
        *reinterpret_cast<float4*>(A.W + w_off + L.g * MB + 8 * s + 2 * L.q) =
            make_float4(f_out * w[s][0], f_out * w[s][2], f_out * w[s][1], f_out * w[s][3]);
      if (c.g == 0) {
        o *= f_out;
        const float res = sqrtf(rs) * f_res;
        if (!(o < FLT_MAX) || !(res < FLT_MAX)) fl |= PRECODE_F_NONFINITE;
        if (A.obj) A.obj[inst] = o;
        if (A.resid) A.resid[inst] = res;
        if (A.flags) A.flags[inst] = fl;
      }
      __syncwarp();  // norm partials read out before the next instance
    }
  }
};

template <int NW, int MINB, bool HOSTIO = false, int MODE = kModeProj>
__global__ void __launch_bounds__(NW * 32, MINB) solve_tch_kernel(SolveArgs A) {
  SolveTCH<NW, HOSTIO, MODE>::run(A);
}

}  // namespace precode
