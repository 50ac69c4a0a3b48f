// Transposed build of the projected-layer tcgen05 kernel (up to 32 users at 256
// antennas).  Thread m of the CTA owns antenna m: column m of W_R = [Re W; Im W]
// (64 values in registers), so each layer's column norm and shrink (the proximal
// step of the projected layer) are thread-local.  The layer in transposed form:
//   residual  D = [H_R hi; H_R lo] [X hi | X lo]^T  (M = N = 128, K = 256 antennas;
//             A the channel tiles, K-major; B the X tiles, MN-major, written by
//             the antenna-owning threads); E = X H'^T - S' from the four blocks
//   update    W^T <- X^T - Q^T E^T,  Q = G'^{-T} conj(H')  (32 x 256 complex,
//             formed once per instance).  A = real form of Q^T, row m =
//             [Re Q[.][m] | Im Q[.][m]] (256 x 64), held in tensor memory as FP16
//             hi / lo (the A operand of tcgen05.mma may come from tensor memory);
//             B = real form of E^T, K-major rows k = [Re E_k | -Im E_k] and k + 32 =
//             [Im E_k | Re E_k], with hi and lo rows stacked to N = 128.  One
//             M = 128 product per antenna half; accumulator lane = antenna, so each
//             thread reads its own column back.
// Against the row build this takes the F = E G'^{-T} product of every layer off
// the CUDA cores (folded into Q once) and the cross-warp column-norm reduction
// (two barriers a layer).
// Q^T is one more product in the setup: D = H_R^T (MN-major A over the same bytes
// as the residual's K-major A) times the real form of G'^{-T} (the row build's
// A_F tiles, each row scaled by its own power of two), M = 128 per antenna half.
// Q is scaled by one power of two g_q (max |g_q Q| in [2^13, 2^14)) before the
// FP16 split, each user's row of E by its own (fsc[k] = 2^-e_k / g_q).  With the
// FP64 orthonormal-basis setup Q = diag(d_u^-2) conj(U'): the same product with
// G'^{-T} replaced by that diagonal.  Units, scales, flags and the setup (Gram
// matrix, register Gauss-Jordan, FP64 fallback, resident factors) are the row
// build's.
#pragma once

#include "solve_tg.cuh"

namespace precode {

struct SolveTGT {
  using G = SolveTG<1>;
  using C = TgCfg;
  using Lane = G::Lane;
  static constexpr int KB = C::KB, MB = C::MB, NT = C::NT, RSF = C::RSF, NC = C::NC;
  static constexpr unsigned FULL = 0xffffffffu;
  static constexpr int ETS = 128;         // residual staging [64 rows of X][128 rows of H_R hi | lo]
  static constexpr uint32_t TM_Q = 384;   // A = Q^T: half h hi at 384 + 64 h, lo at + 32
  static_assert(64 * ETS * 4 <= C::OFF_EC - C::OFF_ED, "the residual staging fits");
  static_assert(MB * 128 * 2 <= C::HS_BYTES, "the X tiles fit the channel area");
  static_assert(TM_Q + 128 <= C::TMEM_COLS && C::TM_E + 128 <= TM_Q, "tensor-memory columns");
  static_assert(C::OFF_FAC % 8 == 0, "the update's two mbarriers sit in the (unused) shrink-factor area");

  // The thread's column of W_R (or X) into the residual's B tiles, [256 antennas]
  // [128] MN-major: columns 0..63 hi, 64..127 lo (consecutive antennas of an access
  // phase write consecutive 16-byte slots)
  __device__ __forceinline__ static void build_xt(const Lane& L, const float (&w)[NC], unsigned char* sm) {
    unsigned char* const base = sm + C::OFF_HS + tc5::tile_off(L.tid, 0, 128);
#pragma unroll
    for (int c = 0; c < NC / 8; ++c) {
      uint4 h, lo;
      G::split8(&w[8 * c], h, lo);
      *reinterpret_cast<uint4*>(base + c * 128) = h;
      *reinterpret_cast<uint4*>(base + (NC / 8 + c) * 128) = lo;
    }
  }

  // D_E = [H_R hi; H_R lo] [X hi | X lo]^T (M = N = 128) over antennas 128 part ..
  // 128 part + 127 (the X tiles of one half of the threads), 8 MMAs
  // (descriptors stepped by their 16-byte address units: a K step is 256 bytes of A,
  // 4096 of B; unrolled, so that the MMAs issue back to back)
  template <int PART>
  __device__ __forceinline__ static void issue_residual(uint32_t tm, uint32_t s_hr, uint32_t s_x) {
    constexpr uint32_t id = tc5::idesc_f16(128, 128, 1);
    const uint64_t a0 = tc5::sdesc(s_hr + PART * 8 * 256, 128, 4096);
    const uint64_t b0 = tc5::sdesc(s_x + PART * 8 * 4096, 2048, 128);
#pragma unroll 4
    for (int ks = 0; ks < 8; ++ks)
      tc5::mma_f16(tm + C::TM_E, a0 + 16 * ks, b0 + 256 * ks, id, PART != 0 || ks != 0);
  }

  // Q^T for antenna half h: D[m][n] = sum_r H_R[r][128 h + m] A_G[n][r] with B =
  // [A_G hi; A_G lo] (N = 128), A = H_R hi, then H_R lo (MN-major), 16 MMAs
  __device__ static void issue_q(uint32_t tm, uint32_t s_hr, uint32_t s_hrl, uint32_t s_ag) {
    constexpr uint32_t id = tc5::idesc_f16(128, 128, 0, 1);
    const uint64_t b0 = tc5::sdesc(s_ag, 128, 1024);
#pragma unroll 1
    for (int h = 0; h < 2; ++h)
#pragma unroll 1
      for (int a = 0; a < 2; ++a) {
        const uint64_t a0 = tc5::sdesc((a ? s_hrl : s_hr) + 2048 * h, 4096, 128);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
          tc5::mma_f16(tm + C::TM_W + 128 * h, a0 + 512 * ks, b0 + 16 * ks, id, (a | ks) != 0);
      }
  }

  // D_W for antenna half h = Q_h^T (tensor memory) times the real form of E^T: A = Q
  // hi against [B_E hi; B_E lo] (N = 128), then A = Q lo against B_E hi (N = 64),
  // three of the four split-FP16 products (lo x lo dropped); each half completes on
  // its own mbarrier, so that its threads start while the other half's MMAs run
  __device__ static void issue_update(uint32_t tm, uint32_t s_be, uint64_t* bar) {
    constexpr uint32_t id = tc5::idesc_f16(128, 128, 0), id64 = tc5::idesc_f16(128, 64, 0);
    const uint64_t b0 = tc5::sdesc(s_be, 128, 1024);
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc5::mma_f16_ta(tm + C::TM_W + 128 * h, tm + TM_Q + 64 * h + 8 * ks, b0 + 16 * ks, id, ks != 0);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks)
        tc5::mma_f16_ta(tm + C::TM_W + 128 * h, tm + TM_Q + 64 * h + 32 + 8 * ks, b0 + 16 * ks, id64, true);
      tc5::commit(smem_addr(bar + h));
    }
  }

  __device__ __forceinline__ static void half_sync(int id) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(NT / 2) : "memory");
  }

  // D_E -> staging: warp w reads TMEM lanes r = 32 (w % 4) + lane (row r of
  // [H_R hi; H_R lo]) and writes St[n][r] = D[r][n] + D[r][n + 64] (X hi and lo
  // summed) for n = 32 (w / 4) + [0, 32)
  __device__ __forceinline__ static void stage_e(const Lane& L, uint32_t tm_q, float* St) {
    const int h = L.w >> 2, r = 32 * (L.w & 3) + L.lane;
    float v1[32], v2[32];
    tc5::ld32x32b_x32(tm_q + C::TM_E + 32 * h, v1);
    tc5::ld32x32b_x32(tm_q + C::TM_E + 64 + 32 * h, v2);
    tc5::wait_ld();
    float* const dst = St + 32 * h * ETS + r;
#pragma unroll
    for (int j = 0; j < 32; ++j) dst[j * ETS] = v1[j] + v2[j];
  }
  // (H hi + H lo) row j times (X hi + X lo) row n, from the staging
  __device__ __forceinline__ static float dpt(const float* St, int j, int n) {
    return St[n * ETS + j] + St[n * ETS + j + 64];
  }

  // The thread's entries E[k][j] (k = 4 w + i, j = lane) minus the targets (diag t',
  // or in the basis S~^T); returns their sum of |E_kj|^2 dinv_j^2
  __device__ __forceinline__ static float form_e(const Lane& L, const float* St, const float* tks,
                                                 const float2* Sx, const float* dinv, bool basis,
                                                 float (&er)[4], float (&ei)[4]) {
    const int k0 = 4 * L.w, j = L.lane;
    const float dj = dinv[j];
    float ss = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = k0 + i;
      er[i] = dpt(St, j, k) - dpt(St, j + 32, k + 32);
      ei[i] = dpt(St, j + 32, k) + dpt(St, j, k + 32);
      if (basis) {
        const float2 s = Sx[k * KB + j];
        er[i] -= s.x;
        ei[i] -= s.y;
      } else if (j == k) {
        er[i] -= tks[k];
      }
      ss += (er[i] * er[i] + ei[i] * ei[i]) * (dj * dj);
    }
    return ss;
  }

  // B_E tiles ([128][64] K-major, hi rows 0..63, lo rows 64..127) from the warp's
  // four rows of E: row k = [Re E_k | -Im E_k], row k + 32 = [Im E_k | Re E_k], each
  // user's row scaled by a power of two into [2^13, 2^14); fsc[k] = 2^-e_k / g_q,
  // the factor D_W's columns k and k + 32 take back
  __device__ __forceinline__ static void make_be(const Lane& L, const float (&er)[4], const float (&ei)[4],
                                                 float gqi, float* fsc, float* Fs, unsigned char* sm) {
    const int k0 = 4 * L.w, j = L.lane;
    float m[4];  // row maxima of |Re|, |Im| (non-negative floats order as their bits)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      m[i] = __uint_as_float(__reduce_max_sync(FULL, __float_as_uint(fmaxf(fabsf(er[i]), fabsf(ei[i])))));
    float* const fw = Fs + L.w * 4 * C::FSS;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      // m in [2^(e-127), 2^(e-126)) for biased exponent e: fs = 2^(140 - e) puts the
      // row into [2^13, 2^14) (e clamped to 26 below), xs = 1 / fs
      float fs = 1.f, xs = 1.f;
      if (m[i] > 0.f && m[i] <= FLT_MAX) {
        const int e = max((int)(__float_as_uint(m[i]) >> 23), 26);
        fs = __uint_as_float((uint32_t)(267 - e) << 23);
        xs = __uint_as_float((uint32_t)(e - 13) << 23);
      }
      if (j == 0) fsc[k0 + i] = xs * gqi;
      fw[i * C::FSS + j] = fs * er[i];
      fw[i * C::FSS + 32 + j] = fs * ei[i];
    }
    __syncwarp();
    {
      // lane (row r = lane % 4, chunk c = lane / 4 of 8 columns of [Re | Im])
      const int r = L.lane & 3, c = L.lane >> 2, k = k0 + r;
      const float4 x0 = *reinterpret_cast<const float4*>(fw + r * C::FSS + 8 * c);
      const float4 x1 = *reinterpret_cast<const float4*>(fw + r * C::FSS + 8 * c + 4);
      const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      uint4 h, lo;
      G::split8(x, h, lo);
      const uint32_t neg = c < 4 ? 0u : 0x80008000u;  // row k: the Im half negated
      *reinterpret_cast<uint4*>(sm + C::OFF_AF + tc5::tile_off(k, 8 * c, 64)) =
          make_uint4(h.x ^ neg, h.y ^ neg, h.z ^ neg, h.w ^ neg);
      *reinterpret_cast<uint4*>(sm + C::OFF_AFL + tc5::tile_off(k, 8 * c, 64)) =
          make_uint4(lo.x ^ neg, lo.y ^ neg, lo.z ^ neg, lo.w ^ neg);
      const int c2 = c < 4 ? c + 4 : c - 4;  // row k + 32 = [Im | Re]
      *reinterpret_cast<uint4*>(sm + C::OFF_AF + tc5::tile_off(k + 32, 8 * c2, 64)) = h;
      *reinterpret_cast<uint4*>(sm + C::OFF_AFL + tc5::tile_off(k + 32, 8 * c2, 64)) = lo;
    }
    __syncwarp();
  }

  // The thread's column of D_W (its antenna's TMEM lane, hi and lo halves summed):
  // SET: w[n] = fsc[n % 32] D[n]; else w[n] -= fsc[n % 32] D[n]
  template <bool SET>
  __device__ __forceinline__ static void read_w(const Lane& L, uint32_t tm_q, const float* fsc, float (&w)[NC]) {
    const uint32_t base = tm_q + C::TM_W + 128 * (L.w >> 2);
    float xs[32];
#pragma unroll
    for (int i = 0; i < 32; i += 4) {
      const float4 f = *reinterpret_cast<const float4*>(fsc + i);
      xs[i] = f.x;
      xs[i + 1] = f.y;
      xs[i + 2] = f.z;
      xs[i + 3] = f.w;
    }
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      float v1[32], v2[32];
      tc5::ld32x32b_x32(base + 32 * p, v1);
      tc5::ld32x32b_x32(base + 64 + 32 * p, v2);
      tc5::wait_ld();
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const float d = v1[j] + v2[j];
        w[32 * p + j] = SET ? xs[j] * d : fmaf(-xs[j], d, w[32 * p + j]);
      }
    }
  }

  // g_q q as FP16 hi / lo pairs (K element 2 i in the low half) into the thread's
  // tensor-memory lane: its row of A = Q^T
  __device__ __forceinline__ static void store_q(const Lane& L, uint32_t tm_q, const float (&q)[NC], float gq) {
    float hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) {
      uint32_t h, l;
      split_h2(gq * q[2 * i], gq * q[2 * i + 1], h, l);
      hi[i] = __uint_as_float(h);
      lo[i] = __uint_as_float(l);
    }
    const uint32_t base = tm_q + TM_Q + 64 * (L.w >> 2);
    tc5::st32x32b_x32(base, hi);
    tc5::st32x32b_x32(base + 32, lo);
    tc5::wait_st();
  }

  // sum of squares of the thread's column in four independent chains
  __device__ __forceinline__ static float sumsq(const float (&w)[NC]) {
    float r[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int n = 0; n < NC; ++n) r[n & 3] = fmaf(w[n], w[n], r[n & 3]);
    return (r[0] + r[1]) + (r[2] + r[3]);
  }

  // Per-user scales d_k (row k's largest component into [1/2, 1)), t' = D t, and the
  // H_R tiles of the scaled channel in one pass over the channel: lane k of warp w
  // holds row k at antennas 32 w .. 32 w + 31 in registers (consecutive lanes read rows
  // 16 bytes apart in the padded layout: distinct bank groups), the eight warps' row
  // maxima meet in pm[8][32]; then it converts as build_hr does
  __device__ static void scale_tiles(const Lane& L, const float2* Hs, float* tks, float* dinv, float* dgs,
                                     float* pm, unsigned char* sm) {
    const int k = L.lane;
    const float4* const src = reinterpret_cast<const float4*>(Hs + k * RSF + 32 * L.w);
    float4 v[16];
    float hm = 0.f;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      v[i] = src[i];
      hm = fmaxf(hm, fmaxf(fmaxf(fabsf(v[i].x), fabsf(v[i].y)), fmaxf(fabsf(v[i].z), fabsf(v[i].w))));
    }
    pm[L.w * KB + k] = hm;
    __syncthreads();
    float rm = pm[k];
#pragma unroll
    for (int q = 1; q < NT / 32; ++q) rm = fmaxf(rm, pm[q * KB + k]);
    const float dg = G::inv_pow2_of(rm);
    if (L.w == 0) {
      tks[k] *= dg;
      dinv[k] = 1.f / dg;
      dgs[k] = dg;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int m0 = 32 * L.w + 8 * c;
      float re[8], im[8];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 x = v[4 * c + i];
        re[2 * i] = dg * x.x;
        im[2 * i] = dg * x.y;
        re[2 * i + 1] = dg * x.z;
        im[2 * i + 1] = dg * x.w;
      }
      uint4 rh, rl, ih, il;
      G::split8(re, rh, rl);
      G::split8(im, ih, il);
      *reinterpret_cast<uint4*>(sm + C::OFF_HR + tc5::tile_off(k, m0, 256)) = rh;
      *reinterpret_cast<uint4*>(sm + C::OFF_HRL + tc5::tile_off(k, m0, 256)) = rl;
      *reinterpret_cast<uint4*>(sm + C::OFF_HR + tc5::tile_off(k + 32, m0, 256)) = ih;
      *reinterpret_cast<uint4*>(sm + C::OFF_HRL + tc5::tile_off(k + 32, m0, 256)) = il;
    }
  }

  __device__ __forceinline__ static float warp_max(float v) {
#pragma unroll
    for (int msk = 1; msk < 32; msk <<= 1) v = fmaxf(v, __shfl_xor_sync(FULL, v, msk));
    return v;
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
    float* const Sg = reinterpret_cast<float*>(sm + C::OFF_ED);  // Gram staging, then St
    double2* const A64 = reinterpret_cast<double2*>(sm + C::OFF_ED);
    float2* const Es = reinterpret_cast<float2*>(sm + C::OFF_ES);
    float* const Fs = reinterpret_cast<float*>(sm + C::OFF_FS);
    float* const np = reinterpret_cast<float*>(sm + C::OFF_NP);
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
    uint64_t* const ubar = reinterpret_cast<uint64_t*>(sm + C::OFF_FAC);  // update halves
    const uint32_t s_x = smem_addr(sm + C::OFF_HS);
    const uint32_t s_hr = smem_addr(sm + C::OFF_HR), s_hrl = smem_addr(sm + C::OFF_HRL);
    const uint32_t s_af = smem_addr(sm + C::OFF_AF);
    if (L.tid == 0) {
      mbar_init(cbar, 1);
      mbar_init(mbar, 1);
      mbar_init(ubar, 1);
      mbar_init(ubar + 1, 1);
    }
    fence_mbar_init();
    if (L.w == 0) tc5::alloc(smem_addr(tslot), C::TMEM_COLS);
    tc5::fence_before_sync();
    __syncthreads();
    tc5::fence_after_sync();
    const uint32_t tm = *tslot;
    const uint32_t tm_q = tm + ((uint32_t)(32 * (L.w & 3)) << 16);  // this warp's lane quarter
    const uint64_t lim = copy_wait_ns(A);

    uint32_t cphase = 0, mphase = 0, uphase = 0;
    const int half = L.w >> 2;  // antenna half of the thread (its update's mbarrier)
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
    // the next channel: thread 0 sets the byte count, then lane j of warp w copies row
    // 4 w + j (j < 4), so that no warp issues more than four copies
    auto issue_copy = [&](int64_t it) {
      if (it >= n_inst || (A.opts & OPT_STALL_COPY)) return;
      int64_t inst, h_off, w_off, t_off;
      int K;
      locate(it, inst, h_off, w_off, t_off, K);
      if (L.tid == 0) {
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(cbar, K * MB * 8);
      }
      __syncthreads();
      const int k = 4 * L.w + L.lane;
      if (L.lane < 4 && k < K) {
        fence_proxy_async_smem();
        bulk_g2s(Hs + k * RSF, A.H + h_off + k * MB, MB * 8, cbar);
      }
    };
    issue_copy(blockIdx.x);
    float w[NC];
#pragma unroll 1
    for (int64_t it = blockIdx.x; it < n_inst; it += gridDim.x) {
      int64_t inst, h_off, w_off, t_off;
      int K;
      locate(it, inst, h_off, w_off, t_off, K);
      if (L.tid == 32 && it + gridDim.x < n_inst && !(A.opts & OPT_STALL_COPY)) {
        // the channel copied at the end of this instance (one contiguous block): into
        // L2 meanwhile
        int64_t i2, h2, w2, t2;
        int K2;
        locate(it + gridDim.x, i2, h2, w2, t2, K2);
        prefetch_l2(A.H + h2, (uint32_t)(K2 * MB * 8));
      }
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
      if (L.tid == NT / 2) bulk_wait_read();  // the last W_T staging is read out
      __syncthreads();

      // ---- per-user scales d_k (H' = D H, applied while converting), t' = D t
      scale_tiles(L, Hs, tks, dinv, dgs, np, sm);

      // ---- Gram matrix G' = H' H'^H (or the resident factor slot's G'^{-T})
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
        G::publish_smem();
        if (L.tid == 0) {
          G::issue_residual(tm, s_hr, s_hr);
          tc5::commit(smem_addr(mbar));
        }
        ok = G::mma_wait(mbar, mphase, lim);
        G::stage_e(L, tm_q, Sg);
      }
      ok = __syncthreads_and(ok) != 0;
      bool singular = false, basis = false;
      {
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
            const float gr = G::dp(Sg, i, j) + G::dp(Sg, i + 32, j + 32);
            const float gi = G::dp(Sg, i + 32, j) - G::dp(Sg, i, j + 32);
            a[c] = (i >= K && i == j) ? make_float2(1.f, 0.f) : make_float2(gr, -gi);
          }
          fast = ok && G::gj_regs(L, a, dsc, rowpub, colpub, A.cond_thr);
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
          G::scale_rows(L, Hs, dgs);
          __syncthreads();
          fl = G::S::template basis_fp64<NT>(L, K, Hs, Es, nullptr, A64, reinterpret_cast<double*>(r64),
                                             reinterpret_cast<double*>(c64), o64, tks);
          singular = (fl & PRECODE_F_SINGULAR) != 0;
          basis = !singular;
          if (basis) {
            const float du = G::row_scale(L, Hs);
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
            G::build_hr(L, Hs, dsc, sm);
          }
        }
      }
      __syncthreads();

      float rss = 0.f, o = 0.f, beta = 1.f, gqi = 1.f;
      bool copied = false;  // the next instance's copy is issued
      if (!singular && ok) {
        // ---- Q^T = H_R^T times the real form of G'^{-T} (basis: of diag(dd))
        {
          const int k0 = 4 * L.w, j = L.lane;
          float fr[4], fi[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int k = k0 + i;
            if (basis) {
              fr[i] = (j == k) ? dd[k] : 0.f;
              fi[i] = 0.f;
            } else {
              const float2 g = Es[k * KB + j];
              fr[i] = g.x;
              fi[i] = g.y;
            }
          }
          G::af_tail(L, fr, fi, fsc, Fs, sm);
        }
        G::publish_smem();
        if (L.tid == 0) {
          issue_q(tm, s_hr, s_hrl, s_af);
          tc5::commit(smem_addr(mbar));
        }
        ok = G::mma_wait(mbar, mphase, lim);
        {
          float q[NC];
          read_w<true>(L, tm_q, fsc, q);  // q = [Re Q[.][m] | Im Q[.][m]]
          float qm = 0.f;
#pragma unroll
          for (int n = 0; n < NC; ++n) qm = fmaxf(qm, fabsf(q[n]));
          qm = warp_max(qm);
          if (L.lane == 0) np[L.w] = qm;
          ok = __syncthreads_and(ok) != 0;
          qm = 0.f;
#pragma unroll
          for (int v = 0; v < NT / 32; ++v) qm = fmaxf(qm, np[v]);
          const float gq = 16384.f * G::inv_pow2_of(qm);
          gqi = 1.f / gq;
          store_q(L, tm_q, q, gq);
          // ---- W^(0)' = S' Q: diag(t') Q, thread-local (the basis below)
#pragma unroll
          for (int k = 0; k < KB; ++k) {
            const float tk = tks[k];
            w[k] = basis ? 0.f : tk * q[k];
            w[KB + k] = basis ? 0.f : tk * q[KB + k];
          }
        }
        if (basis) {  // W^(0)' = -E_0 Q with E_0 = -S~^T', one update with X = 0
          {
            const int k0 = 4 * L.w, j = L.lane;
            float er[4], ei[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const float2 sv = Es[(k0 + i) * KB + j];
              er[i] = -sv.x;
              ei[i] = -sv.y;
            }
            make_be(L, er, ei, gqi, fsc, Fs, sm);
          }
          G::publish_smem();
          // issued by a thread of the second half: the first half's warps go on meanwhile
          if (L.tid == NT / 2) issue_update(tm, s_af, ubar);
          ok = G::mma_wait(ubar + half, uphase, lim) && ok;
          read_w<false>(L, tm_q, fsc, w);
        }
        // global scale b: max(|W^(0)'|, |targets|) into [8, 16)
        float wm = 0.f;
#pragma unroll
        for (int i = 0; i < NC; ++i) wm = fmaxf(wm, fabsf(w[i]));
        if (basis)
          for (int idx = L.tid; idx < KB * KB; idx += NT)
            wm = fmaxf(wm, fmaxf(fabsf(Es[idx].x), fabsf(Es[idx].y)));
        if (L.tid < KB) wm = fmaxf(wm, fabsf(tks[L.tid]));
        wm = warp_max(wm);
        if (L.lane == 0) wred[L.w] = wm;
        ok = __syncthreads_and(ok) != 0;
        wm = 0.f;
#pragma unroll
        for (int v = 0; v < NT / 32; ++v) wm = fmaxf(wm, wred[v]);
        beta = 16.f * G::inv_pow2_of(wm);
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

        // ---- layers (scaled units).  Each antenna half waits for its own half of
        // the update, shrinks and writes its X tiles; the residual's MMAs over the
        // first half's antennas start while the second half is still at work.
        const int T = A.T;
        bool pending = false;  // an update of W is in flight
#pragma unroll 1
        for (int l = 0; l < T; ++l) {
          const float tau = fmaxf(__ldg(A.step + l), 0.f) * beta, tau2 = tau * tau;
          if (pending) {
            ok = G::mma_wait(ubar + half, uphase, lim) && ok;
            read_w<false>(L, tm_q, fsc, w);
          }
          const float r2 = sumsq(w);
          const float f = r2 > tau2 ? 1.f - tau * rsqrtf(r2) : 0.f;
#pragma unroll
          for (int n = 0; n < NC; ++n) w[n] *= f;
          build_xt(L, w, sm);
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          tc5::fence_before_sync();
          if (half == 0) {
            half_sync(1);
            if (L.tid == 0) {
              tc5::fence_after_sync();
              issue_residual<0>(tm, s_hr, s_x);
            }
          }
          ok = __syncthreads_and(ok) != 0;
          tc5::fence_after_sync();
          if (L.tid == 0) {
            issue_residual<1>(tm, s_hr, s_x);
            tc5::commit(smem_addr(mbar));
          }
          ok = G::mma_wait(mbar, mphase, lim) && ok;
          stage_e(L, tm_q, Sg);
          ok = __syncthreads_and(ok) != 0;
          pending = false;
          if (!ok) break;
          {
            float er[4], ei[4];
            form_e(L, Sg, tks, Es, dinv, basis, er, ei);
            make_be(L, er, ei, gqi, fsc, Fs, sm);
          }
          G::publish_smem();
          // issued by a thread of the second half: the first half's warps go on meanwhile
          if (L.tid == NT / 2) issue_update(tm, s_af, ubar);
          pending = true;
        }
        if (pending) {
          ok = G::mma_wait(ubar + half, uphase, lim) && ok;
          read_w<false>(L, tm_q, fsc, w);
        }

        // ---- objective (sum of the column norms) and residual of W_T
        o = sqrtf(sumsq(w));
        ok = __syncthreads_and(ok) != 0;
        if (A.resid && ok) {
          if (basis) {  // against the channel itself: H' again, and its tiles
            for (int idx = L.tid; idx < K * (MB / 2); idx += NT) {
              const int k = idx / (MB / 2), m2 = idx % (MB / 2);
              *reinterpret_cast<float4*>(Hs + k * RSF + 2 * m2) =
                  *reinterpret_cast<const float4*>(A.H + h_off + k * MB + 2 * m2);
            }
            __syncthreads();
            G::build_hr(L, Hs, dgs, sm);
            __syncthreads();
          }
          build_xt(L, w, sm);
          G::publish_smem();
          if (L.tid == 0) {
            issue_residual<0>(tm, s_hr, s_x);
            issue_residual<1>(tm, s_hr, s_x);
            tc5::commit(smem_addr(mbar));
          }
          ok = G::mma_wait(mbar, mphase, lim) && ok;
          stage_e(L, tm_q, Sg);
          ok = __syncthreads_and(ok) != 0;
          if (ok) {  // the X tiles are read: the channel area takes the next copy
            issue_copy(it + gridDim.x);
            copied = true;
          }
          float er[4], ei[4];
          rss = form_e(L, Sg, tks, Es, dinv, false, er, ei);
        }
      }
      // every MMA has completed (or timed out) on every thread: the channel area
      // takes the next instance's copy (if not yet issued)
      ok = __syncthreads_and(ok) != 0;
      if (ok && !copied) issue_copy(it + gridDim.x);
      {  // W_T (or 0) as [K][256] float2 into the channel-tile area (read by no MMA any
         // more), written back below by one bulk copy
        const float fo = 1.f / beta;
        const bool zero = singular || !ok;
        float2* const ws = reinterpret_cast<float2*>(sm + C::OFF_HR) + L.tid;
#pragma unroll
        for (int k = 0; k < KB; ++k)
          if (k < K) ws[k * MB] = zero ? make_float2(0.f, 0.f) : make_float2(fo * w[k], fo * w[KB + k]);
        fence_proxy_async_smem();
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
      if (L.tid == NT / 2) {  // W_T out: one contiguous block of K rows
        bulk_s2g(A.W + w_off, sm + C::OFF_HR, (uint32_t)(K * MB * 8));
        bulk_commit();
      }
      float rs = 0.f, ob = 0.f;  // warp 0: the eight warps' sums
      if (L.w == 0) {
        rs = L.lane < NT / 32 ? wred[L.lane] : 0.f;
        ob = L.lane < NT / 32 ? np[L.lane] : 0.f;
#pragma unroll
        for (int msk = 1; msk < NT / 32; msk <<= 1) {
          rs += __shfl_xor_sync(FULL, rs, msk);
          ob += __shfl_xor_sync(FULL, ob, msk);
        }
      }
      if (L.tid == 0) {
        if (singular) {  // W = 0: objective 0, residual ||S||_F
          ob = 0.f;
          rs = 0.f;
          for (int k = 0; k < KB; ++k) rs += (tks[k] * dinv[k]) * (tks[k] * dinv[k]);
        }
        const float fo = 1.f / beta;
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
      __syncthreads();  // the scalars are read out
      if (!ok) break;   // a tensor-core wait ran out: stop (TMEM is freed below)
    }
    if (L.tid == NT / 2) bulk_wait();  // the last W_T write-back has completed
    tc5::fence_before_sync();
    __syncthreads();
    if (L.w == 0) tc5::dealloc(tm, C::TMEM_COLS);
  }
};

__global__ void __launch_bounds__(TgCfg::NT, 1) solve_tgt_kernel(SolveArgs A) { SolveTGT::run(A); }

}  // namespace precode
