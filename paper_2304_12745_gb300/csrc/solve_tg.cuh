// Projected-layer solve kernel for up to 32 users at 256 antennas on the
// fifth-generation tensor cores: both layer contractions are tcgen05.mma
// (kind::f16, split FP16, FP32 accumulators in tensor memory), issued by one
// thread with both operands in shared memory.
//
// Real form.  Rows 0..31 hold the real parts of the 32 (padded) users, rows
// 32..63 the imaginary parts: W_R = [Re W; Im W] (64 x 256), H_R = [Re H'; Im H'].
//   residual  D_E = W_R H_R^T   (M = 64, N = 64, K = 256 antennas):
//             Re E[k][j] = D[k][j] - D[k+32][j+32],  Im E[k][j] = D[k][j+32] + D[k+32][j]
//   update    D_W = A_F H_R     (M = 64, N = 256, K = 64),  A_F = [[Re F, Im F], [Im F, -Re F]]
//             is [Re; Im] of F conj(H'), with F = (E - S') G'^{-T};  W <- X - D_W
// The same H_R bytes serve as the K-major B of the residual and the MN-major B
// of the update.  Each product takes three MMAs per K step (hi x lo, lo x hi,
// hi x hi), the split-FP16 scheme of the warp-MMA kernels, in the same exact
// power-of-two units: per-user channel scales (H' = D H, t' = D t) and one global
// scale b on W and the targets.  F has no a-priori range, so each user's row of F
// is scaled by its own power of two into [2^13, 2^14) before the FP16 split and
// that row of D_W scaled back (exact in FP32).
//
// One CTA of eight warps per instance, persistent over instances (one CTA per
// SM).  The residual runs as M = N = 128: A = [W_R hi; W_R lo] and B = [H_R hi;
// H_R lo] are each one contiguous 64-row pair of tiles, and the four blocks of
// the product summed give (W hi + W lo)(H hi + H lo)^T, split FP16 in 16 MMAs
// (the lo x lo block only adds accuracy).  The update keeps M = 64 (three
// passes): with M = 64 the accumulator row r sits in TMEM lane 32 (r / 16) +
// r % 16, and warp w may read lanes 32 (w % 4) .. + 31, so warps w and w + 4
// read rows 16 (w % 4) .. + 15, lane l the row 16 (w % 4) + l % 16 at columns
// 128 (w / 4) + 64 (l / 16) + [0, 64) of D_W, which is also the part of W the
// thread keeps in registers across the layers.  The CUDA cores form the column
// norms and the shrink (registers, shuffles, shared memory), the FP16 operand
// tiles and F (lane = column of E, four rows per warp, so that row and column
// operands come as broadcasts and consecutive words); the tensor cores do the
// two contractions.  Shared-memory mappings are chosen so that the eight lanes
// of each 16-byte access phase hit distinct bank groups.
// Setup: the Gram matrix as a residual with A = B = H_R, the equilibrated
// Gauss-Jordan inverse of the multi-warp kernels held in registers (four entries
// a thread, the pivot row and column published through shared memory, one
// barrier a pivot; the pivot spread is the condition estimate) or, above the
// threshold, their FP64 orthonormal-basis path (U over the channel, each row of U
// scaled by a power of two like H', G'^{-T} replaced by those scales, targets
// S~^T); W^(0) is the update with X = 0.
#pragma once

#include <cfloat>

#include "f16mma.cuh"
#include "solve_tcw.cuh"
#include "tcgen05.cuh"

namespace precode {

struct TgCfg {
  static constexpr int KB = 32, MB = 256, NT = 256, RSF = MB + 2;
  static constexpr int NC = 64;  // W columns per thread
  // shared memory (bytes)
  static constexpr int OFF_HS = 0;         // raw channel [32][258] float2 (setup); layers: A_W hi | lo
  static constexpr int HS_BYTES = 66560;
  static constexpr int OFF_AWL = 32768;    // A_W lo inside the channel area
  static constexpr int OFF_HR = OFF_HS + HS_BYTES;  // H_R hi [64][256] FP16; end: W staging
  static constexpr int OFF_HRL = OFF_HR + 32768;    // H_R lo
  static constexpr int OFF_AF = OFF_HRL + 32768;    // A_F hi [64][64] FP16
  static constexpr int OFF_AFL = OFF_AF + 8192;     // A_F lo
  static constexpr int EDS = 68;                    // staging row stride (floats)
  static constexpr int OFF_ED = OFF_AFL + 8192;     // residual staging [128][EDS]; setup: FP64 matrix
  static constexpr int ECS = KB + 1;                    // E row stride (float2)
  static constexpr int OFF_EC = OFF_ED + 128 * EDS * 4;  // E [32][33] float2
  static constexpr int OFF_ES = OFF_EC + KB * ECS * 8;   // G'^{-T} or S~^T [32][32] float2
  static constexpr int FSS = 72;                         // F staging row stride (floats)
  static constexpr int OFF_FS = OFF_ES + 8192;           // F staging [8 warps][4 rows][FSS]
  static constexpr int OFF_NP = OFF_FS + 8 * 4 * FSS * 4;  // column-norm partials [4 row groups][256]
  static constexpr int OFF_FAC = OFF_NP + 4096;          // shrink factors [256]
  static constexpr int OFF_S64 = OFF_FAC + 1024;         // FP64 pivots: double2[32] x 2, double[32]
  // t[32] dsc[32] misc[8] wred[8] fsc[32] dd[32] dgs[32] rowpub[2][2][32] colpub[2][2][32] (float2)
  static constexpr int OFF_SC = OFF_S64 + 1280;
  static constexpr int SC_BYTES = 2752;
  static constexpr int OFF_DINV = OFF_SC + SC_BYTES;
  static constexpr int OFF_BAR = OFF_DINV + 128;         // copy barrier, MMA barrier, TMEM address
  static constexpr int SMEM_BYTES = OFF_BAR + 32;
  static constexpr uint32_t TMEM_COLS = 512;
  static constexpr uint32_t TM_W = 0, TM_E = 256;  // D_W: M = 64, 256 columns; D_E: M = 128, 128 columns
  static_assert(KB * RSF * 8 <= HS_BYTES && OFF_AWL + 32768 <= HS_BYTES, "channel and A_W share an area");
  static_assert(128 * EDS * 4 >= KB * KB * 16, "the FP64 matrix of the setup fits the staging");
  static_assert(OFF_HR % 1024 == 0 && OFF_AF % 128 == 0 && OFF_ED % 16 == 0 && OFF_ES % 16 == 0 &&
                    OFF_FS % 16 == 0 && OFF_SC % 16 == 0 && OFF_BAR % 8 == 0,
                "alignment");
  static_assert(SMEM_BYTES <= 227 * 1024, "one CTA per SM");
};

template <int MINB>
struct SolveTG {
  using C = TgCfg;
  using S = SolveTCW<kModeProj, 4, 256>;  // FP64 setup helper (run with NT threads), padded rows
  using Lane = typename S::Lane;
  static constexpr int KB = C::KB, MB = C::MB, NT = C::NT, RSF = C::RSF, NC = C::NC, ECS = C::ECS,
                       EDS = C::EDS;
  static constexpr unsigned FULL = 0xffffffffu;
  static_assert(S::RSF == RSF && S::KB == KB && S::MB == MB, "the setup helper's geometry");

  __device__ __forceinline__ static float inv_pow2_of(float v) {
    if (!(v > 0.f) || !(v <= FLT_MAX)) return 1.f;
    int ex;
    frexpf(v, &ex);
    return ldexpf(1.f, -ex);
  }

  // eight floats -> hi and lo FP16 chunks of 16 bytes
  __device__ __forceinline__ static void split8(const float* x, uint4& hi, uint4& lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) split_h2(x[2 * i], x[2 * i + 1], h[i], l[i]);
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
  }

  // Power-of-two scale putting each padded channel row's largest component into
  // [1/2, 1) (1 for a zero row): thread (row tid / 8, 16-byte chunks tid % 8 + 8 i),
  // so that the eight threads of an access phase read consecutive chunks.  Every
  // thread of the row gets the row's scale.
  __device__ static float row_scale(const Lane& L, const float2* Hs) {
    const int k = L.tid >> 3, p = L.tid & 7;
    const float4* row = reinterpret_cast<const float4*>(Hs + k * RSF);
    float hm = 0.f;
#pragma unroll 8
    for (int i = 0; i < MB / 16; ++i) {
      const float4 v = row[p + 8 * i];
      hm = fmaxf(hm, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
    }
    hm = fmaxf(hm, __shfl_xor_sync(FULL, hm, 1));
    hm = fmaxf(hm, __shfl_xor_sync(FULL, hm, 2));
    hm = fmaxf(hm, __shfl_xor_sync(FULL, hm, 4));
    return inv_pow2_of(hm);
  }
  // rows of Hs times rs[k], in place (same mapping)
  __device__ static void scale_rows(const Lane& L, float2* Hs, const float* rs) {
    const int k = L.tid >> 3, p = L.tid & 7;
    float4* row = reinterpret_cast<float4*>(Hs + k * RSF);
    const float f = rs[k];
#pragma unroll 8
    for (int i = 0; i < MB / 16; ++i) {
      const float4 v = row[p + 8 * i];
      row[p + 8 * i] = make_float4(f * v.x, f * v.y, f * v.z, f * v.w);
    }
  }

  // H_R hi / lo from the padded channel rows times rs[k] (exact powers of two):
  // warp w converts antennas 32 w .. 32 w + 31, lane k row k (Re into tile row k,
  // Im into row k + 32), so that an access phase covers eight rows
  __device__ static void build_hr(const Lane& L, const float2* Hs, const float* rs, unsigned char* sm) {
    const int k = L.lane;
    const float f = rs[k];
#pragma unroll 1
    for (int c = 0; c < 4; ++c) {
      const int m0 = 32 * L.w + 8 * c;
      const float4* src = reinterpret_cast<const float4*>(Hs + k * RSF + m0);
      float re[8], im[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 v = src[i];
        re[2 * i] = f * v.x;
        im[2 * i] = f * v.y;
        re[2 * i + 1] = f * v.z;
        im[2 * i + 1] = f * v.w;
      }
      uint4 rh, rl, ih, il;
      split8(re, rh, rl);
      split8(im, ih, il);
      *reinterpret_cast<uint4*>(sm + C::OFF_HR + tc5::tile_off(k, m0, 256)) = rh;
      *reinterpret_cast<uint4*>(sm + C::OFF_HRL + tc5::tile_off(k, m0, 256)) = rl;
      *reinterpret_cast<uint4*>(sm + C::OFF_HR + tc5::tile_off(k + 32, m0, 256)) = ih;
      *reinterpret_cast<uint4*>(sm + C::OFF_HRL + tc5::tile_off(k + 32, m0, 256)) = il;
    }
  }

  // row and first column of the thread's part of W (64 columns)
  __device__ __forceinline__ static int w_row(const Lane& L) { return 16 * (L.w & 3) + (L.lane & 15); }
  __device__ __forceinline__ static int w_col(const Lane& L) {
    return 128 * (L.w >> 2) + 64 * (L.lane >> 4);
  }

  // The thread's 64 entries of W_R (or X) into the residual's A tiles (hi, lo)
  __device__ __forceinline__ static void build_aw(const Lane& L, const float (&w)[NC], unsigned char* sm) {
    const int r = w_row(L), c0 = w_col(L);
#pragma unroll
    for (int c = 0; c < NC / 8; ++c) {
      uint4 h, lo;
      split8(&w[8 * c], h, lo);
      *reinterpret_cast<uint4*>(sm + C::OFF_HS + tc5::tile_off(r, c0 + 8 * c, 256)) = h;
      *reinterpret_cast<uint4*>(sm + C::OFF_AWL + tc5::tile_off(r, c0 + 8 * c, 256)) = lo;
    }
  }

  // D_E = [A hi; A lo] [H_R hi; H_R lo]^T (M = N = 128, both K-major), 16 MMAs
  // (descriptors stepped by their 16-byte address units; unrolled, so that the MMAs
  // issue back to back)
  __device__ static void issue_residual(uint32_t tm, uint32_t a, uint32_t b) {
    constexpr uint32_t id = tc5::idesc_f16(128, 128, 0);
    const uint64_t a0 = tc5::sdesc(a, 128, 4096), b0 = tc5::sdesc(b, 128, 4096);
#pragma unroll
    for (int ks = 0; ks < 16; ++ks) tc5::mma_f16(tm + C::TM_E, a0 + 16 * ks, b0 + 16 * ks, id, ks != 0);
  }
  // D_W = A_F[64][64] (K-major) H_R[64][256] (MN-major), split FP16: 3 x 4 MMAs
  __device__ static void issue_update(uint32_t tm, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                      uint32_t b_lo) {
    constexpr uint32_t id = tc5::idesc_f16(64, 256, 1);
    const uint32_t as[3] = {a_hi, a_lo, a_hi}, bs[3] = {b_lo, b_hi, b_hi};
#pragma unroll
    for (int ps = 0; ps < 3; ++ps) {
      const uint64_t a0 = tc5::sdesc(as[ps], 128, 1024), b0 = tc5::sdesc(bs[ps], 4096, 128);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) tc5::mma_f16(tm + C::TM_W, a0 + 16 * ks, b0 + 512 * ks, id, (ps | ks) != 0);
    }
  }

  // D_E -> staging: warp w reads TMEM lanes 32 (w % 4) + lane = rows r of [A hi;
  // A lo] and writes S[r][n] = D[r][n] + D[r][n + 64] (H_R hi and lo columns
  // summed) for n = 32 (w / 4) + [0, 32)
  __device__ __forceinline__ static void stage_e(const Lane& L, uint32_t tm_q, float* Sg) {
    const int h = L.w >> 2, r = 32 * (L.w & 3) + L.lane;
    float v1[32], v2[32];
    tc5::ld32x32b_x32(tm_q + C::TM_E + 32 * h, v1);
    tc5::ld32x32b_x32(tm_q + C::TM_E + 64 + 32 * h, v2);
    tc5::wait_ld();
    float* dst = Sg + r * EDS + 32 * h;
#pragma unroll
    for (int j = 0; j < 32; j += 4)
      *reinterpret_cast<float4*>(dst + j) =
          make_float4(v1[j] + v2[j], v1[j + 1] + v2[j + 1], v1[j + 2] + v2[j + 2], v1[j + 3] + v2[j + 3]);
  }
  // (A hi + A lo) row r times (H hi + H lo) row n, from the staging
  __device__ __forceinline__ static float dp(const float* Sg, int r, int n) {
    return Sg[r * EDS + n] + Sg[(r + 64) * EDS + n];
  }

  // The thread's entries E[k][j] (k = 4 w + i, j = lane) from the staging, minus
  // the targets (diag t', or in the basis S~^T); returns their sum of
  // |E_kj|^2 dinv_j^2
  __device__ __forceinline__ static float form_e(const Lane& L, const float* Sg, const float* tks,
                                                 const float2* St, const float* dinv, bool basis,
                                                 float (&er)[4], float (&ei)[4]) {
    const int k0 = 4 * L.w, j = L.lane;
    const float dj = dinv[j];
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + i;
      er[i] = dp(Sg, k, j) - dp(Sg, k + 32, j + 32);
      ei[i] = dp(Sg, k, j + 32) + dp(Sg, k + 32, j);
      if (basis) {
        const float2 s = St[k * KB + j];
        er[i] -= s.x;
        ei[i] -= s.y;
      } else if (j == k) {
        er[i] -= tks[k];
      }
      ss += (er[i] * er[i] + ei[i] * ei[i]) * (dj * dj);
    }
    return ss;
  }

  // F from the thread's E entries (F = E G'^{-T}, or in the basis F = E diag(dd)),
  // each row's power-of-two range scale (into fsc: the factor D_W's rows k and
  // k + 32 take back), and the thread's entries of A_F hi / lo.  The warp's rows
  // of E meet in Ec (warp-synchronous): row operands are broadcasts, G'^{-T} rows
  // consecutive words.
  // With tdiag (the start, E_0 = -diag(t')): F_0[k][j] = -t'_k G'^{-T}[k][j] directly.
  __device__ __forceinline__ static void make_af(const Lane& L, const float (&er)[4], const float (&ei)[4],
                                                 bool basis, const float* dd, const float2* G, float2* Ec,
                                                 float* fsc, float* Fs, unsigned char* sm,
                                                 const float* tdiag = nullptr) {
    const int k0 = 4 * L.w, j = L.lane;
    float fr[4], fi[4];
    if (tdiag) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float2 g = G[(k0 + i) * KB + j];
        const float tk = tdiag[k0 + i];
        fr[i] = -tk * g.x;
        fi[i] = -tk * g.y;
      }
    } else if (basis) {
      const float d = dd[j];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        fr[i] = er[i] * d;
        fi[i] = ei[i] * d;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        Ec[(k0 + i) * ECS + j] = make_float2(er[i], ei[i]);
        fr[i] = fi[i] = 0.f;
      }
      __syncwarp();
#pragma unroll 8
      for (int l = 0; l < KB; ++l) {
        const float2 g = G[l * KB + j];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 e = Ec[(k0 + i) * ECS + l];
          fr[i] = fmaf(e.x, g.x, fmaf(-e.y, g.y, fr[i]));
          fi[i] = fmaf(e.x, g.y, fmaf(e.y, g.x, fi[i]));
        }
      }
      __syncwarp();
    }
    af_tail(L, fr, fi, fsc, Fs, sm);
  }

  // The warp's four rows of F (k = 4 w + i, column j = lane), each scaled by its
  // own power of two into [2^13, 2^14) (fsc[k]: the factor that rows k and k + 32
  // of the product take back), into the A_F tiles hi / lo
  __device__ __forceinline__ static void af_tail(const Lane& L, const float (&fr)[4], const float (&fi)[4],
                                                 float* fsc, float* Fs, unsigned char* sm) {
    const int k0 = 4 * L.w, j = L.lane;
    float m[4];  // row maxima of |Re|, |Im| (non-negative floats order as their bits)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      m[i] = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(fmaxf(fabsf(fr[i]), fabsf(fi[i])))));
    // scaled F rows [Re F | Im F] into the warp's FP32 staging (word stores), then
    // lane (row r = lane % 4, chunk c = lane / 4 of 8 columns) splits 8 columns and
    // writes them into rows k (chunk c) and k + 32 (chunk c +- 4, Re negated) of the
    // A_F tiles with 16-byte stores (an access phase spans four rows)
    float* const fw = Fs + L.w * 4 * C::FSS;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + i;
      // max |F_k| into [2^13, 2^14): with m in [2^(e-127), 2^(e-126)) for biased
      // exponent e, fs = 2^(140 - e) (e clamped to 26 below), xs = 1 / fs
      float fs = 1.f, xs = 1.f;
      if (m[i] > 0.f && m[i] <= FLT_MAX) {
        const int e = max((int)(__float_as_uint(m[i]) >> 23), 26);
        fs = __uint_as_float((uint32_t)(267 - e) << 23);
        xs = __uint_as_float((uint32_t)(e - 13) << 23);
      }
      if (j == 0) fsc[k] = xs;
      fw[i * C::FSS + j] = fs * fr[i];
      fw[i * C::FSS + 32 + j] = fs * fi[i];
    }
    __syncwarp();
    {
      const int r = L.lane & 3, c = L.lane >> 2, k = k0 + r;
      const float4 x0 = *reinterpret_cast<const float4*>(fw + r * C::FSS + 8 * c);
      const float4 x1 = *reinterpret_cast<const float4*>(fw + r * C::FSS + 8 * c + 4);
      const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      uint4 h, lo;
      split8(x, h, lo);
      *reinterpret_cast<uint4*>(sm + C::OFF_AF + tc5::tile_off(k, 8 * c, 64)) = h;
      *reinterpret_cast<uint4*>(sm + C::OFF_AFL + tc5::tile_off(k, 8 * c, 64)) = lo;
      // row k + 32 = [Im F | -Re F]: chunk c of [Re | Im] lands at c + 4 (negated) or c - 4
      const int c2 = c < 4 ? c + 4 : c - 4;
      const uint32_t neg = c < 4 ? 0x80008000u : 0u;
      const uint4 hn = make_uint4(h.x ^ neg, h.y ^ neg, h.z ^ neg, h.w ^ neg);
      const uint4 ln = make_uint4(lo.x ^ neg, lo.y ^ neg, lo.z ^ neg, lo.w ^ neg);
      *reinterpret_cast<uint4*>(sm + C::OFF_AF + tc5::tile_off(k + 32, 8 * c2, 64)) = hn;
      *reinterpret_cast<uint4*>(sm + C::OFF_AFL + tc5::tile_off(k + 32, 8 * c2, 64)) = ln;
    }
    __syncwarp();
  }

  // w = a w - xs D_W for the thread's 64 entries (a = 1, or 0 for W^(0))
  __device__ __forceinline__ static void apply_update(const Lane& L, uint32_t tm_q, const float* fsc,
                                                      float a, float (&w)[NC]) {
    const float xs = fsc[w_row(L) & 31];
    const uint32_t base = tm_q + C::TM_W + 128 * (L.w >> 2);
#pragma unroll
    for (int c = 0; c < NC; c += 32) {
      float v[32];
      tc5::ld16x2_x32<64>(base + c, v);
      tc5::wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) w[c + j] = fmaf(-xs, v[j], a * w[c + j]);
    }
  }

  template <int HALF>
  __device__ __forceinline__ static void rs_step(float* v, int b, int mask) {
#pragma unroll
    for (int j = 0; j < HALF; ++j) {
      const float send = b ? v[j] : v[j + HALF];
      const float keep = b ? v[j + HALF] : v[j];
      v[j] = keep + __shfl_xor_sync(FULL, send, mask);
    }
  }

  // Squared column norms over all 64 rows: each warp sums its 16 rows of the
  // lane's 64 columns (reduce-scatter over the 16 lanes of the half, 32 columns
  // at a time), the four row groups' partials meet in shared memory; thread t
  // then owns column t and writes f(r2) for it into fac.  ok is and-ed over the
  // CTA (uniform on return).  Returns sqrt(r2) of the thread's column.
  template <class Fn>
  __device__ __forceinline__ static float colnorms(const Lane& L, const float (&w)[NC], float* np,
                                                   float* fac, Fn f, bool& ok) {
    const int b3 = (L.lane >> 3) & 1, b2 = (L.lane >> 2) & 1, b1 = (L.lane >> 1) & 1, b0 = L.lane & 1;
    float* dst = np + (L.w & 3) * 256 + w_col(L) + 16 * b3 + 8 * b2 + 4 * b1 + 2 * b0;
#pragma unroll
    for (int c = 0; c < NC / 32; ++c) {
      float v[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) v[j] = w[32 * c + j] * w[32 * c + j];
      rs_step<16>(v, b3, 8);
      rs_step<8>(v, b2, 4);
      rs_step<4>(v, b1, 2);
      rs_step<2>(v, b0, 1);
      *reinterpret_cast<float2*>(dst + 32 * c) = make_float2(v[0], v[1]);
    }
    ok = __syncthreads_and(ok) != 0;
    const float r = (np[L.tid] + np[256 + L.tid]) + (np[512 + L.tid] + np[768 + L.tid]);
    fac[L.tid] = f(r);
    __syncthreads();
    return sqrtf(r);
  }

  // a s - f b (complex a, f, b; real s): one entry of an elimination step
  __device__ __forceinline__ static float2 sfb(float2 a, float s, float2 f, float2 b) {
    return make_float2(fmaf(f.y, b.y, fmaf(-f.x, b.x, s * a.x)), fmaf(-f.y, b.x, fmaf(-f.x, b.y, s * a.y)));
  }
  __device__ __forceinline__ static float2 cscale(float2 c, float r) { return make_float2(c.x * r, c.y * r); }

  // Equilibrated Gauss-Jordan inverse (no pivoting; pivot spread max d / min d of
  // the equilibrated matrix is the condition estimate) with the matrix in
  // registers: thread (i = tid / 8, columns j_c = tid % 8 + 8 c) holds a[c] =
  // G'^T[i][j_c] on entry and G'^{-T}[i][j_c] on a true return.  Pivot p takes
  // every entry to a s_i - f_i A[p][j] (row p: s = 1 / A[p][p], f = 0; any other
  // row: s = 1, f = A[i][p] / A[p][p]), then sets column p to the inverse's
  // (1 / A[p][p] at the pivot, -f_i elsewhere): the in-place elimination.  Two
  // pivots per barrier: the rows and columns of pivots p and p + 1 are published by
  // their owners (two alternating buffers), and each thread replays pivot p on the
  // entries pivot p + 1 reads (row p + 1 at its columns, its row's column p + 1, the
  // pivot) before applying p + 1 to its own: the entries of the one-pivot-a-step
  // elimination, in half the barriers.
  __device__ static bool gj_regs(const Lane& L, float2 (&a)[4], float* dsc, float2* rowpub,
                                 float2* colpub, float cond_thr) {
    const int i = L.tid >> 3, j0 = L.tid & 7;
    if (j0 == (i & 7)) {  // the diagonal entry (static register indices only)
      float dv = a[0].x;
#pragma unroll
      for (int c = 1; c < 4; ++c)
        if (c == (i >> 3)) dv = a[c].x;
      dsc[i] = rsqrtf(dv);
    }
    __syncthreads();
    const float di = dsc[i];
    float dj[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      dj[c] = dsc[j0 + 8 * c];
      a[c] = cscale(a[c], di * dj[c]);
    }
    bool fail = false;
    float dmin = FLT_MAX, dmax = 0.f;
#pragma unroll 1
    for (int p = 0; p < KB; p += 2) {
      const int q = p + 1;
      float2* const rp = rowpub + 2 * KB * ((p >> 1) & 1);  // rows p, q: [2][KB]
      float2* const cp = colpub + 2 * KB * ((p >> 1) & 1);  // columns p, q: [2][KB]
      if (i == p || i == q)
#pragma unroll
        for (int c = 0; c < 4; ++c) rp[(i - p) * KB + j0 + 8 * c] = a[c];
      if (j0 == (p & 7) || j0 == (q & 7)) {
        const int cc = (j0 == (p & 7)) ? (p >> 3) : (q >> 3);
        float2 v = a[0];
#pragma unroll
        for (int c = 1; c < 4; ++c)
          if (c == cc) v = a[c];
        cp[(j0 == (p & 7) ? 0 : KB) + i] = v;
      }
      __syncthreads();
      const float2* const Rp = rp;
      const float2* const Rq = rp + KB;
      // pivot p
      const float dp = Rp[p].x;
      fail |= !(dp > 0.f) || !(dp < FLT_MAX);
      dmin = fminf(dmin, dp);
      dmax = fmaxf(dmax, dp);
      const float invp = rcp_nr(dp);
      const float2 cip = cp[i], ciq = cp[KB + i];
      float2 rpb[4], rqb[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        rpb[c] = Rp[j0 + 8 * c];
        rqb[c] = Rq[j0 + 8 * c];
      }
      const float2 aqp = Rq[p], apq = Rp[q], aqq = Rq[q];
      const bool ip = i == p, iq = i == q;
      const int colp = (j0 == (p & 7)) ? (p >> 3) : -1, colq = (j0 == (q & 7)) ? (q >> 3) : -1;
      const float sp = ip ? invp : 1.f;
      const float2 fp = ip ? make_float2(0.f, 0.f) : cscale(cip, invp);
      // what pivot q reads, after pivot p: its row at my columns, my row's column q, its pivot
      const float2 fq = cscale(aqp, invp);
      float2 bq[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        bq[c] = sfb(rqb[c], 1.f, fq, rpb[c]);
        if (c == colp) bq[c] = make_float2(-fq.x, -fq.y);
        a[c] = sfb(a[c], sp, fp, rpb[c]);
        if (c == colp) a[c] = ip ? make_float2(invp, 0.f) : make_float2(-fp.x, -fp.y);
      }
      const float2 cq = sfb(ciq, sp, fp, apq);
      const float dq = fmaf(fq.y, apq.y, fmaf(-fq.x, apq.x, aqq.x));
      // pivot q
      fail |= !(dq > 0.f) || !(dq < FLT_MAX);
      dmin = fminf(dmin, dq);
      dmax = fmaxf(dmax, dq);
      const float invq = rcp_nr(dq);
      const float sq = iq ? invq : 1.f;
      const float2 fqq = iq ? make_float2(0.f, 0.f) : cscale(cq, invq);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        a[c] = sfb(a[c], sq, fqq, bq[c]);
        if (c == colq) a[c] = iq ? make_float2(invq, 0.f) : make_float2(-fqq.x, -fqq.y);
      }
    }
    const bool ok = !fail && !(dmax > cond_thr * dmin);
    if (ok)
#pragma unroll
      for (int c = 0; c < 4; ++c) a[c] = cscale(a[c], di * dj[c]);
    return ok;
  }

  __device__ __forceinline__ static bool mbar_try(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
  }

  // wait for the MMAs' commit (bounded by lim and an iteration count)
  __device__ static bool mma_wait(uint64_t* bar, uint32_t& phase, uint64_t lim) {
    bool ok = mbar_try(bar, phase);
    if (!ok) {
      const uint64_t t0 = global_ns();
      for (uint32_t i = 1; i < (1u << 24) && !ok; ++i) {
        ok = mbar_try(bar, phase);
        if (!ok && (i & 31) == 0 && global_ns() - t0 > lim) break;
      }
    }
    phase ^= 1u;
    tc5::fence_after_sync();
    return ok;
  }

  // all threads' generic shared-memory writes visible to the tensor cores and
  // their earlier TMEM loads complete, then the issuing thread may start MMAs
  __device__ __forceinline__ static void publish_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
  }

  __device__ static void run(const SolveArgs& A) {
    extern __shared__ __align__(1024) unsigned char sm[];
    Lane L;
    L.tid = threadIdx.x;
    L.w = L.tid >> 5;
    L.lane = L.tid & 31;
    L.g = L.lane >> 2;
    L.q = L.lane & 3;
    float2* const Hs = reinterpret_cast<float2*>(sm + C::OFF_HS);
    float* const Ws = reinterpret_cast<float*>(sm + C::OFF_HR);
    float* const Sg = reinterpret_cast<float*>(sm + C::OFF_ED);
    double2* const A64 = reinterpret_cast<double2*>(sm + C::OFF_ED);
    float2* const Ec = reinterpret_cast<float2*>(sm + C::OFF_EC);
    float2* const Es = reinterpret_cast<float2*>(sm + C::OFF_ES);
    float* const Fs = reinterpret_cast<float*>(sm + C::OFF_FS);
    float* const np = reinterpret_cast<float*>(sm + C::OFF_NP);
    float* const fac = reinterpret_cast<float*>(sm + C::OFF_FAC);
    double2* const r64 = reinterpret_cast<double2*>(sm + C::OFF_S64);
    double2* const c64 = r64 + KB;
    double* const o64 = reinterpret_cast<double*>(c64 + KB);
    float* const tks = reinterpret_cast<float*>(sm + C::OFF_SC);
    float* const dsc = tks + KB;
    int* const misc = reinterpret_cast<int*>(dsc + KB);
    float* const wred = reinterpret_cast<float*>(misc + 8);
    float* const fsc = wred + 8;
    float* const dd = fsc + KB;
    float* const dgs = dd + KB;
    float2* const rowpub = reinterpret_cast<float2*>(dgs + KB);
    float2* const colpub = rowpub + 4 * KB;
    float* const dinv = reinterpret_cast<float*>(sm + C::OFF_DINV);
    uint64_t* const cbar = reinterpret_cast<uint64_t*>(sm + C::OFF_BAR);
    uint64_t* const mbar = cbar + 1;
    uint32_t* const tslot = reinterpret_cast<uint32_t*>(cbar + 2);
    const uint32_t s_aw = smem_addr(sm + C::OFF_HS);
    const uint32_t s_hr = smem_addr(sm + C::OFF_HR), s_hrl = smem_addr(sm + C::OFF_HRL);
    const uint32_t s_af = smem_addr(sm + C::OFF_AF), s_afl = smem_addr(sm + C::OFF_AFL);
    if (L.tid == 0) {
      mbar_init(cbar, 1);
      mbar_init(mbar, 1);
    }
    fence_mbar_init();
    if (L.w == 0) tc5::alloc(smem_addr(tslot), C::TMEM_COLS);
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tm = *tslot;
    const uint32_t tm_q = tm + ((uint32_t)(32 * (L.w & 3)) << 16);  // this warp's lane quarter
    const uint64_t lim = copy_wait_ns(A);

    uint32_t cphase = 0, mphase = 0;
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
    auto issue_copy = [&](int64_t it) {
      if (L.tid != 0 || it >= n_inst || (A.opts & OPT_STALL_COPY)) return;
      int64_t inst, h_off, w_off, t_off;
      int K;
      locate(it, inst, h_off, w_off, t_off, K);
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(cbar, K * MB * 8);
      for (int k = 0; k < K; ++k) bulk_g2s(Hs + k * RSF, A.H + h_off + k * MB, MB * 8, cbar);
    };
    issue_copy(blockIdx.x);
    float w[NC];
#pragma unroll 1
    for (int64_t it = blockIdx.x; it < n_inst; it += gridDim.x) {
      int64_t inst, h_off, w_off, t_off;
      int K;
      locate(it, inst, h_off, w_off, t_off, K);
      if (L.tid < KB) tks[L.tid] = L.tid < K ? A.t[t_off + L.tid] : 0.f;
      if (L.tid == 0) misc[0] = mbar_wait_bounded(cbar, cphase, lim) ? 1 : 0;
      __syncthreads();
      if (misc[0] == 0) {
        if (L.tid == 0) {
          atomicAdd(A.err, 1ull);
          if (A.flags) A.flags[inst] = PRECODE_F_TIMEOUT;
          misc[1] = mbar_wait_bounded(cbar, cphase, lim) ? 1 : 0;
        }
        __syncthreads();
        if (misc[1] == 0) break;  // the copy never landed: stop (TMEM is freed below)
        cphase ^= 1u;
        __syncthreads();
        issue_copy(it + gridDim.x);
        continue;
      }
      if (L.tid != 0) mbar_wait_bounded(cbar, cphase, lim);  // completed: returns at once
      cphase ^= 1u;
      if (K < KB) {  // padded users: zero channel rows
        for (int idx = L.tid; idx < (KB - K) * MB; idx += NT)
          Hs[(K + idx / MB) * RSF + idx % MB] = make_float2(0.f, 0.f);
      }
      __syncthreads();

      // ---- per-user scales d_k (H' = D H, applied while converting), t' = D t
      {
        const float dg = row_scale(L, Hs);
        if ((L.tid & 7) == 0) {
          const int k = L.tid >> 3;
          tks[k] *= dg;
          dinv[k] = 1.f / dg;
          dgs[k] = dg;
        }
      }
      __syncthreads();
      build_hr(L, Hs, dgs, sm);

      // ---- Gram matrix G' = H' H'^H as a residual with A = B = H_R (or the
      // resident factor slot's G'^{-T}, when it holds the FP32 path's)
      int fl = 0;
      bool ok = true;
      const float2* fin = nullptr;
      float2* fout = nullptr;
      if (A.fac) {
        if (A.opts & OPT_FAC_EXPORT)
          fout = A.fac + inst * (int64_t)fac_stride(KB);
        else if (A.fidx && A.fidx[inst] >= 0)
          fin = A.fac + A.fidx[inst];
      }
      const bool imported = fin && fin[KB * KB].x == 1.f;
      if (!imported) {
        publish_smem();
        if (L.tid == 0) {
          issue_residual(tm, s_hr, s_hr);
          tc5::commit(smem_addr(mbar));
        }
        ok = mma_wait(mbar, mphase, lim);
        stage_e(L, tm_q, Sg);
      }
      ok = __syncthreads_and(ok) != 0;
      bool singular = false, basis = false;
      {
        // thread (i, j_c) takes G'^T[i][j_c] = conj(G'[i][j_c]); padded users get a unit pivot
        const int i = L.tid >> 3, j0 = L.tid & 7;
        float2 a[4];
        bool fast = imported;
        if (imported) {
#pragma unroll
          for (int c = 0; c < 4; ++c) a[c] = fin[i * KB + j0 + 8 * c];
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            const int j = j0 + 8 * c;
            const float gr = dp(Sg, i, j) + dp(Sg, i + 32, j + 32);
            const float gi = dp(Sg, i + 32, j) - dp(Sg, i, j + 32);
            a[c] = (i >= K && i == j) ? make_float2(1.f, 0.f) : make_float2(gr, -gi);
          }
          fast = ok && gj_regs(L, a, dsc, rowpub, colpub, A.cond_thr);
        }
        if (fout && ok) {
#pragma unroll
          for (int c = 0; c < 4; ++c) fout[i * KB + j0 + 8 * c] = a[c];
          if (L.tid == 0) fout[KB * KB] = make_float2(fast ? 1.f : 0.f, 0.f);
        }
        if (fast) {
#pragma unroll
          for (int c = 0; c < 4; ++c) Es[i * KB + j0 + 8 * c] = a[c];
        } else if (ok) {
          // FP64 path on the scaled channel H' (in place), then U's rows scaled by
          // powers of two (U' = D_u U): S~^T columns times d_u, dd = d_u^-2
          scale_rows(L, Hs, dgs);
          __syncthreads();
          fl = S::template basis_fp64<NT>(L, K, Hs, Es, nullptr, A64, reinterpret_cast<double*>(r64),
                                          reinterpret_cast<double*>(c64), o64, tks);
          singular = (fl & PRECODE_F_SINGULAR) != 0;
          basis = !singular;
          if (basis) {
            const float du = row_scale(L, Hs);
            if ((L.tid & 7) == 0) {
              dd[L.tid >> 3] = 1.f / (du * du);
              dsc[L.tid >> 3] = du;
            }
            __syncthreads();
            for (int idx = L.tid; idx < KB * KB; idx += NT) {
              const float sc = dsc[idx % KB];
              const float2 v = Es[idx];
              Es[idx] = make_float2(sc * v.x, sc * v.y);
            }
            build_hr(L, Hs, dsc, sm);
          }
        }
      }
      __syncthreads();

      float rss = 0.f, o = 0.f, beta = 1.f;
      if (!singular && ok) {
        // ---- W^(0)' = -F_0 conj(H') with E_0 = -S' (X = 0)
        {
          const int k0 = 4 * L.w, j = L.lane;
          float er[4], ei[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (basis) {
              const float2 sv = Es[(k0 + i) * KB + j];
              er[i] = -sv.x;
              ei[i] = -sv.y;
            } else {
              er[i] = (j == k0 + i) ? -tks[k0 + i] : 0.f;
              ei[i] = 0.f;
            }
          }
          make_af(L, er, ei, basis, dd, Es, Ec, fsc, Fs, sm, basis ? nullptr : tks);
        }
        publish_smem();
        if (L.tid == 0) {
          issue_update(tm, s_af, s_afl, s_hr, s_hrl);
          tc5::commit(smem_addr(mbar));
        }
        ok = mma_wait(mbar, mphase, lim);
#pragma unroll
        for (int i = 0; i < NC; ++i) w[i] = 0.f;
        apply_update(L, tm_q, fsc, 0.f, w);
        // global scale b: max(|W^(0)'|, |targets|) into [8, 16)
        float wm = 0.f;
#pragma unroll
        for (int i = 0; i < NC; ++i) wm = fmaxf(wm, fabsf(w[i]));
        if (basis)
          for (int idx = L.tid; idx < KB * KB; idx += NT)
            wm = fmaxf(wm, fmaxf(fabsf(Es[idx].x), fabsf(Es[idx].y)));
        if (L.tid < KB) wm = fmaxf(wm, fabsf(tks[L.tid]));
#pragma unroll
        for (int msk = 1; msk < 32; msk <<= 1) wm = fmaxf(wm, __shfl_xor_sync(FULL, wm, msk));
        if (L.lane == 0) wred[L.w] = wm;
        ok = __syncthreads_and(ok) != 0;
        wm = 0.f;
#pragma unroll
        for (int q = 0; q < NT / 32; ++q) wm = fmaxf(wm, wred[q]);
        beta = 16.f * inv_pow2_of(wm);
#pragma unroll
        for (int i = 0; i < NC; ++i) w[i] *= beta;
        __syncthreads();  // every read of wred, t' and S~^T done
        if (L.tid < KB) tks[L.tid] *= beta;
        if (basis)
          for (int idx = L.tid; idx < KB * KB; idx += NT) {
            const float2 sv = Es[idx];
            Es[idx] = make_float2(beta * sv.x, beta * sv.y);
          }
        __syncthreads();

        // ---- layers (scaled units)
        const int T = A.T;
#pragma unroll 1
        for (int l = 0; l < T; ++l) {
          const float tau = fmaxf(__ldg(A.step + l), 0.f) * beta, tau2 = tau * tau;
          colnorms(L, w, np, fac, [&](float r2) { return r2 > tau2 ? 1.f - tau * rsqrtf(r2) : 0.f; },
                   ok);
          if (!ok) break;
          const float* fr = fac + w_col(L);
#pragma unroll
          for (int i = 0; i < NC; i += 4) {
            const float4 f4 = *reinterpret_cast<const float4*>(fr + i);
            w[i] *= f4.x;
            w[i + 1] *= f4.y;
            w[i + 2] *= f4.z;
            w[i + 3] *= f4.w;
          }
          build_aw(L, w, sm);
          publish_smem();
          if (L.tid == 0) {
            issue_residual(tm, s_aw, s_hr);
            tc5::commit(smem_addr(mbar));
          }
          ok = mma_wait(mbar, mphase, lim) && ok;
          stage_e(L, tm_q, Sg);
          ok = __syncthreads_and(ok) != 0;
          {
            float er[4], ei[4];
            form_e(L, Sg, tks, Es, dinv, basis, er, ei);
            make_af(L, er, ei, basis, dd, Es, Ec, fsc, Fs, sm);
          }
          publish_smem();
          if (L.tid == 0) {
            issue_update(tm, s_af, s_afl, s_hr, s_hrl);
            tc5::commit(smem_addr(mbar));
          }
          ok = mma_wait(mbar, mphase, lim) && ok;
          apply_update(L, tm_q, fsc, 1.f, w);
        }

        // ---- objective and residual of W_T
        o = colnorms(L, w, np, fac, [](float) { return 0.f; }, ok);
        if (A.resid && ok) {
          if (basis) {  // against the channel itself: H' again, and its tiles
            for (int idx = L.tid; idx < K * (MB / 2); idx += NT) {
              const int k = idx / (MB / 2), m2 = idx % (MB / 2);
              *reinterpret_cast<float4*>(Hs + k * RSF + 2 * m2) =
                  *reinterpret_cast<const float4*>(A.H + h_off + k * MB + 2 * m2);
            }
            __syncthreads();
            build_hr(L, Hs, dgs, sm);
            __syncthreads();
          }
          build_aw(L, w, sm);
          publish_smem();
          if (L.tid == 0) {
            issue_residual(tm, s_aw, s_hr);
            tc5::commit(smem_addr(mbar));
          }
          ok = mma_wait(mbar, mphase, lim) && ok;
          stage_e(L, tm_q, Sg);
          __syncthreads();
          float er[4], ei[4];
          rss = form_e(L, Sg, tks, Es, dinv, false, er, ei);
        }
      }
      // every MMA has completed (or timed out) on every thread: the channel
      // area takes the next instance's copy, H_R the staging of W_T'
      ok = __syncthreads_and(ok) != 0;
      if (ok) issue_copy(it + gridDim.x);
      {
        const int r = w_row(L), c0 = w_col(L);
#pragma unroll
        for (int i = 0; i < NC; i += 4) {  // 16-byte chunk (c0 + i) / 4, XOR-swizzled by row
          const int ch = ((c0 + i) >> 2) ^ (r & 7);
          *reinterpret_cast<float4*>(Ws + r * MB + 4 * ch) =
              (singular || !ok) ? make_float4(0.f, 0.f, 0.f, 0.f)
                                : make_float4(w[i], w[i + 1], w[i + 2], w[i + 3]);
        }
      }
#pragma unroll
      for (int msk = 1; msk < 32; msk <<= 1) {
        rss += __shfl_xor_sync(FULL, rss, msk);
        o += __shfl_xor_sync(FULL, o, msk);
      }
      if (L.lane == 0) {
        wred[L.w] = rss;
        np[L.w] = o;
      }
      __syncthreads();
      const float fo = 1.f / beta;
      for (int k = L.tid >> 7; k < K; k += 2) {  // thread t: antennas 2 (t % 128) + {0, 1}
        const int m = 2 * (L.tid & 127);
        const int col = 4 * ((m >> 2) ^ (k & 7)) + (m & 3);
        const float2 re = *reinterpret_cast<const float2*>(Ws + k * MB + col);
        const float2 im = *reinterpret_cast<const float2*>(Ws + (k + 32) * MB + col);
        *reinterpret_cast<float4*>(A.W + w_off + k * MB + m) =
            make_float4(fo * re.x, fo * im.x, fo * re.y, fo * im.y);
      }
      if (L.tid == 0) {
        float rs = 0.f, ob = 0.f;
        for (int q = 0; q < NT / 32; ++q) {
          rs += wred[q];
          ob += np[q];
        }
        if (singular) {  // W = 0: objective 0, residual ||S||_F
          ob = 0.f;
          rs = 0.f;
          for (int k = 0; k < KB; ++k) rs += (tks[k] * dinv[k]) * (tks[k] * dinv[k]);
        }
        ob *= fo;
        const float res = sqrtf(rs) * fo;
        if (!ok) {
          atomicAdd(A.err, 1ull);
          fl |= PRECODE_F_TIMEOUT;
        }
        if (!(ob < FLT_MAX) || !(res < FLT_MAX)) fl |= PRECODE_F_NONFINITE;
        if (A.obj) A.obj[inst] = ob;
        if (A.resid) A.resid[inst] = res;
        if (A.flags) A.flags[inst] = fl;
      }
      __syncthreads();  // the staging and the scalars are read out
      if (!ok) break;   // a tensor-core wait ran out: stop (TMEM is freed below)
    }
    tc5::fence_before_sync();
    __syncthreads();
    if (L.w == 0) tc5::dealloc(tm, C::TMEM_COLS);
  }
};

template <int MINB>
__global__ void __launch_bounds__(TgCfg::NT, MINB) solve_tg_kernel(SolveArgs A) {
  SolveTG<MINB>::run(A);
}

}  // namespace precode
