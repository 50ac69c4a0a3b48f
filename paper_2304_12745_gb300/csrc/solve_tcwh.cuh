// Multi-warp projected-layer solve kernel with the layers' two big contractions
// as split-FP16 warp MMAs (m16n8k16): the residual E = W H^T and the update
// W -= F conj(H), for buckets of up to KB = 8 KW users at exactly MB antennas.
// Everything else is the split-TF32 multi-warp kernel's: one CTA of KW warps per
// instance, warp w owning users 8w .. 8w + 7 over all antennas in the m16n8
// accumulator order, the raw channel in shared memory (FP32, rows padded by 16
// bytes) for the split-TF32 setup, F = E G^{-T} as split-TF32 MMAs, the Gram
// inverse and the FP64 path, user padding.  For the layers each channel row is
// converted once per instance, in place, into 16-byte chunks per antenna pair
// (Re hi, Im hi, Re lo, Im lo as FP16 pairs), permuted within each group of 8
// chunks by a row-dependent XOR so that both the residual's reads (8 users x 4
// antenna pairs per quarter warp) and the update's (4 user pairs x 1 antenna
// pair) hit 8 distinct bank groups.
//
// FP16 covers a narrow exponent range, so the instance is solved in units made
// of exact powers of two, under which the projected iteration is equivariant:
// with D = diag(d_k) and a scalar b,
//   H' = D H,  t'_k = b d_k t_k,  W' = b W,  mu' = b mu,  G' = D G D,
//   E' = W' H'^T - S' = b E D,  F' = E' G'^{-T} = b E G^{-T} D^{-1},  F' conj(H') = b E Q;
// d_k puts the largest component of user k's channel row in [1/2, 1) (a weak
// user's row stays out of FP16's subnormals) and b puts max(|W^(0)'|, t') in
// [8, 16).  F' has no cheap a-priori bound (it grows with the Gram condition), so
// each warp checks its F' tiles every layer: past 2^14 it moves a power of two
// from F' to the channel operand of its update (F' 2^-s times 2^s conj(H'),
// exact, s <= 15); past 2^29 that layer's update runs as split TF32 in FP32
// range instead.  Instances on the FP64 path (equilibrated Gram condition above
// the threshold) run all their layers as split TF32: at such conditions the
// iterates carry rounding far above FP32's and may leave FP16's range.  W, the
// objective and the residual (per column d_k^{-1}) are scaled back on the way out.
#pragma once

#include "f16mma.cuh"
#include "solve_tcw.cuh"

namespace precode {

template <int KW, int MB_>
struct TcwhCfg : TcwCfg<KW, MB_> {
  using B = TcwCfg<KW, MB_>;
  // the split-TF32 kernel's layout plus d_k^{-1} [KB] after its scalars
  static constexpr int OFF_DINV = B::OFF_SC + B::SC_BYTES;
  static constexpr int OFF_BAR = align_up(OFF_DINV + B::KB * 4, 16);
  static constexpr int SMEM_BYTES = align_up(OFF_BAR + 8, 16);
};

template <int KW, int MB_>
struct SolveTCWH : SolveTCW<kModeProj, KW, MB_> {
  using S = SolveTCW<kModeProj, KW, MB_>;
  using C = TcwhCfg<KW, MB_>;
  using Lane = typename S::Lane;
  using WT = typename S::WT;
  static constexpr int KB = S::KB, MB = S::MB, NS = S::NS, NT = S::NT, RSF = S::RSF, NQ = S::NQ;
  static constexpr unsigned FULL = 0xffffffffu;
  static constexpr float FMAX = 16384.f;  // bound on |F'| entries fed to the FP16 update

  __device__ __forceinline__ static float inv_pow2_of(float v) {
    if (!(v > 0.f) || !(v <= FLT_MAX)) return 1.f;
    int ex;
    frexpf(v, &ex);
    return ldexpf(1.f, -ex);
  }

  // ---- FP16 chunk layout of the scaled channel
  static constexpr int RC = RSF / 2;  // chunks per row (MB / 2 + the padding chunk)
  // bank-group swizzle of row u: user pairs and row parity spread over the 8 groups
  __device__ __forceinline__ static int hsw(int u) { return ((u >> 1) & 3) | ((u & 1) << 2); }
  // position within its row of chunk p (antennas 2p, 2p + 1) of row u: bank group
  // (u RC + pos) mod 8 = (p ^ hsw(u)) mod 8, since MB / 2 is a multiple of 8
  __device__ __forceinline__ static int chunk_pos(int u, int p) {
    return (p & ~7) | ((((p ^ hsw(u)) & 7) - u) & 7);
  }

  // In place: raw FP32 rows -> FP16 chunks.  One thread per (row, group of 8
  // chunks) reads its group whole before writing it back permuted.
  __device__ static void to_chunks(const Lane& L, float2* Hs) {
    constexpr int NG = MB / 16;
    uint4* const hc = reinterpret_cast<uint4*>(Hs);
    const float4* const hr = reinterpret_cast<const float4*>(Hs);
    for (int idx = L.tid; idx < KB * NG; idx += NT) {
      const int u = idx / NG, g8 = 8 * (idx % NG);
      float4 v[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = hr[u * RC + g8 + j];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        uint32_t rh, rl, ih, il;
        split_h2(v[j].x, v[j].z, rh, rl);  // Re H', antennas 2p, 2p + 1
        split_h2(v[j].y, v[j].w, ih, il);  // Im H'
        hc[u * RC + chunk_pos(u, g8 + j)] = make_uint4(rh, ih, rl, il);
      }
    }
  }

  // E' tile ct of the warp's rows from FP16 halves of W' and the channel chunks,
  // 16 antennas per MMA; A = (Re W, Im W) rows throughout, products with Re H'
  // into ar, with Im H' into ai:  E_re = [ar]_g - [ai]_g+8,  E_im = [ai]_g + [ar]_g+8.
  __device__ __forceinline__ static void e_tile_c(const Lane& L, const float2* Hs, const WT& w,
                                                  int ct, float (&e)[4]) {
    float ar[2][4], ai[2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) ar[i][k] = ai[i][k] = 0.f;
    const int u = 8 * ct + L.g;
    const uint4* const row = reinterpret_cast<const uint4*>(Hs) + u * RC;
    const uint4* const r0 = row + chunk_pos(u, L.q);      // blocks s even: pair 4s + q
    const uint4* const r1 = row + chunk_pos(u, 4 + L.q);  // blocks s odd
#pragma unroll
    for (int s = 0; s < NS; s += 2) {
      uint32_t ah[4], al[4];
      split_h2_ordered(w[s][0], w[s][1], ah[0], al[0]);          // Re W, block s
      split_h2_ordered(w[s][2], w[s][3], ah[1], al[1]);          // Im W, block s
      split_h2_ordered(w[s + 1][0], w[s + 1][1], ah[2], al[2]);  // Re W, block s + 1
      split_h2_ordered(w[s + 1][2], w[s + 1][3], ah[3], al[3]);  // Im W, block s + 1
      const uint4 c0 = r0[4 * s], c1 = r1[4 * s];                // pairs 4s + q, 4s + 4 + q
      float (&r)[4] = ar[(s >> 1) & 1];
      float (&i)[4] = ai[(s >> 1) & 1];
      mma_f16(r, ah[0], ah[1], ah[2], ah[3], c0.z, c1.z);
      mma_f16(i, ah[0], ah[1], ah[2], ah[3], c0.w, c1.w);
      mma_f16(r, al[0], al[1], al[2], al[3], c0.x, c1.x);
      mma_f16(i, al[0], al[1], al[2], al[3], c0.y, c1.y);
      mma_f16(r, ah[0], ah[1], ah[2], ah[3], c0.x, c1.x);
      mma_f16(i, ah[0], ah[1], ah[2], ah[3], c0.y, c1.y);
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

  // W' -= F' conj(H') with FP16 halves: A from the warp's F' tile kt (rows g:
  // (-F_re, +F_im), rows g + 8: (-F_im, -F_re) over users 8kt + {0..7}); B = the
  // conj(H') entries of users 8kt + 2q, 8kt + 2q + 1 at antenna 8nt + g, taken from
  // the two users' chunks with byte permutes (times xs when SCALED).
  template <bool SCALED>
  __device__ __forceinline__ static void update_c(const Lane& L, const float2* Hs, const float4* ft,
                                                  float xs, WT& w) {
    const uint32_t sel = (L.g & 1) ? 0x7632u : 0x5410u;  // the antenna's half of each pair
    const __half2 xs2 = __float2half2_rn(xs);
#pragma unroll 1
    for (int kt = 0; kt < KW; ++kt) {
      const float4 f = ft[kt * 32 + L.lane];
      uint32_t h01, l01, h23, l23;
      split_h2_ordered(f.x, f.y, h01, l01);
      split_h2_ordered(f.z, f.w, h23, l23);
      const uint32_t nh01 = neg_h2(h01), nl01 = neg_h2(l01), nh23 = neg_h2(h23), nl23 = neg_h2(l23);
      const int u0 = 8 * kt + 2 * L.q, u1 = u0 + 1;
      const uint4* const row0 = reinterpret_cast<const uint4*>(Hs) + u0 * RC;
      const uint4* const row1 = row0 + RC;
      const int pe = L.g >> 1, po = 4 + (L.g >> 1);  // pair within a group of 8, nt even / odd
      const uint4* const a0 = row0 + chunk_pos(u0, pe);
      const uint4* const a1 = row0 + chunk_pos(u0, po);
      const uint4* const b0 = row1 + chunk_pos(u1, pe);
      const uint4* const b1 = row1 + chunk_pos(u1, po);
#pragma unroll
      for (int nt = 0; nt < NS; ++nt) {
        const uint4 c0 = (nt & 1) ? a1[8 * (nt >> 1)] : a0[8 * (nt >> 1)];
        const uint4 c1 = (nt & 1) ? b1[8 * (nt >> 1)] : b0[8 * (nt >> 1)];
        uint32_t rh = __byte_perm(c0.x, c1.x, sel), ih = __byte_perm(c0.y, c1.y, sel) ^ 0x80008000u;
        uint32_t rl = __byte_perm(c0.z, c1.z, sel), il = __byte_perm(c0.w, c1.w, sel) ^ 0x80008000u;
        if constexpr (SCALED) {
          rh = h2_bits(__hmul2(*reinterpret_cast<const __half2*>(&rh), xs2));
          ih = h2_bits(__hmul2(*reinterpret_cast<const __half2*>(&ih), xs2));
          rl = h2_bits(__hmul2(*reinterpret_cast<const __half2*>(&rl), xs2));
          il = h2_bits(__hmul2(*reinterpret_cast<const __half2*>(&il), xs2));
        }
        mma_f16(w[nt], nh01, nh23, h23, nh01, rl, il);
        mma_f16(w[nt], nl01, nl23, l23, nl01, rh, ih);
        mma_f16(w[nt], nh01, nh23, h23, nh01, rh, ih);
      }
    }
  }

  // The same update as split TF32 in FP32 range, for an F' beyond the FP16
  // update's reach: conj(H') rebuilt from the chunks (hi + lo).
  __device__ __forceinline__ static void update_c_tf32(const Lane& L, const float2* Hs, const float4* ft,
                                                       WT& w) {
    const int hsel = L.g & 1;
    auto part = [&](uint32_t hi, uint32_t lo) {
      const __half2 a = *reinterpret_cast<const __half2*>(&hi), b = *reinterpret_cast<const __half2*>(&lo);
      return hsel ? __high2float(a) + __high2float(b) : __low2float(a) + __low2float(b);
    };
#pragma unroll 1
    for (int kt = 0; kt < KW; ++kt) {
      const float4 f = ft[kt * 32 + L.lane];
      uint32_t c0h, c0l, c1h, c1l, c2h, c2l, c3h, c3l;
      split_tf32_ordered(f.x, c0h, c0l);
      split_tf32_ordered(f.y, c1h, c1l);
      split_tf32_ordered(f.z, c2h, c2l);
      split_tf32_ordered(f.w, c3h, c3l);
      const uint32_t n0h = neg_bits(c0h), n1h = neg_bits(c1h), n2h = neg_bits(c2h), n3h = neg_bits(c3h);
      const uint32_t n0l = neg_bits(c0l), n1l = neg_bits(c1l), n2l = neg_bits(c2l), n3l = neg_bits(c3l);
      const int u0 = 8 * kt + 2 * L.q, u1 = u0 + 1;
      const uint4* const row0 = reinterpret_cast<const uint4*>(Hs) + u0 * RC;
      const uint4* const row1 = row0 + RC;
#pragma unroll
      for (int nt = 0; nt < NS; ++nt) {
        const int p = 4 * nt + (L.g >> 1);
        const uint4 c0 = row0[chunk_pos(u0, p)], c1 = row1[chunk_pos(u1, p)];
        uint32_t r0h, r0l, r1h, r1l, i0h, i0l, i1h, i1l;
        split_tf32_ordered(part(c0.x, c0.z), r0h, r0l);
        split_tf32_ordered(part(c1.x, c1.z), r1h, r1l);
        split_tf32_ordered(-part(c0.y, c0.w), i0h, i0l);
        split_tf32_ordered(-part(c1.y, c1.w), i1h, i1l);
        mma_tf32(w[nt], n0h, n2h, n1h, n3h, r0l, r1l);
        mma_tf32(w[nt], c2h, n0h, c3h, n1h, i0l, i1l);
        mma_tf32(w[nt], n0l, n2l, n1l, n3l, r0h, r1h);
        mma_tf32(w[nt], c2l, n0l, c3l, n1l, i0h, i1h);
        mma_tf32(w[nt], n0h, n2h, n1h, n3h, r0h, r1h);
        mma_tf32(w[nt], c2h, n0h, c3h, n1h, i0h, i1h);
      }
    }
  }

  // E' tile by tile (FP16 chunks), F' = E' G'^{-T} accumulated by split-TF32 MMAs, then
  // the F' range check of the warp: returns the channel factor xs for the FP16
  // update (1, or 2^s with F' stored scaled by 2^-s), or 0 when F' is beyond
  // what the FP16 update can take (F' stored as is, for the split-TF32 update).
  __device__ __forceinline__ static float residual_fh(const Lane& L, const float2* Hs, const float4* gf,
                                                      const float* tks, const WT& w, float4* ft) {
    float fa[KW][4];
#pragma unroll
    for (int i = 0; i < KW; ++i)
#pragma unroll
      for (int k = 0; k < 4; ++k) fa[i][k] = 0.f;
#pragma unroll 1
    for (int ct = 0; ct < KW; ++ct) {
      float e[4];
      e_tile_c(L, Hs, w, ct, e);
      S::sub_s(L, tks, ct, e);
      uint32_t c0h, c0l, c1h, c1l, c2h, c2l, c3h, c3l;
      split_tf32_ordered(e[0], c0h, c0l);
      split_tf32_ordered(e[1], c1h, c1l);
      split_tf32_ordered(e[2], c2h, c2l);
      split_tf32_ordered(e[3], c3h, c3l);
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
    }
    float fm = 0.f;
#pragma unroll
    for (int cp = 0; cp < KW; ++cp)
#pragma unroll
      for (int k = 0; k < 4; ++k) fm = fmaxf(fm, fabsf(fa[cp][k]));
#pragma unroll
    for (int msk = 1; msk < 32; msk <<= 1) fm = fmaxf(fm, __shfl_xor_sync(FULL, fm, msk));
    float fs = 1.f, xs = 1.f;
    if (fm > FMAX && fm <= FLT_MAX) {  // move 2^s from F' to the channel operand
      int ex;
      frexpf(fm, &ex);
      const int s = ex - 14;
      if (s > 15) {
        xs = 0.f;  // |2^s conj(H')| would leave FP16: split-TF32 update
      } else {
        fs = ldexpf(1.f, -s);
        xs = ldexpf(1.f, s);
      }
    }
#pragma unroll
    for (int cp = 0; cp < KW; ++cp)
      ft[cp * 32 + L.lane] = make_float4(fs * fa[cp][0], fs * fa[cp][1], fs * fa[cp][2], fs * fa[cp][3]);
    __syncwarp();
    return xs;
  }

  // ||E||_F^2 over the lane's entries in original units (columns d_k^{-1}, then
  // the 1 / b applied by the caller); E' from the FP16 chunks or (TF32) split-TF32
  // MMAs on the raw channel
  template <bool TF32>
  __device__ __forceinline__ static float residual_ssh(const Lane& L, const float2* Hs, const float* tks,
                                                       const float* dinv, const WT& w) {
    float ss = 0.f;
#pragma unroll 1
    for (int ct = 0; ct < KW; ++ct) {
      float e[4];
      if constexpr (TF32)
        S::template e_tile<false>(L, Hs, w, ct, e);
      else
        e_tile_c(L, Hs, w, ct, e);
      S::sub_s(L, tks, ct, e);
      const float d0 = dinv[8 * ct + 2 * L.q], d1 = dinv[8 * ct + 2 * L.q + 1];
      ss += d0 * d0 * (e[0] * e[0] + e[2] * e[2]) + d1 * d1 * (e[1] * e[1] + e[3] * e[3]);
    }
    return ss;
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
    float* const dinv = reinterpret_cast<float*>(smem + C::OFF_DINV);
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

      // ---- per-user scales: row 8w + g of H' = d H (in place), t' = d t
      {
        float2* const hr = Hs + (8 * L.w + L.g) * RSF + 2 * L.q;
        float hm = 0.f;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          const float4 v = *reinterpret_cast<const float4*>(hr + 8 * s);
          hm = fmaxf(hm, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        hm = fmaxf(hm, __shfl_xor_sync(FULL, hm, 1));  // the 4 lanes of the row
        hm = fmaxf(hm, __shfl_xor_sync(FULL, hm, 2));
        const float dg = inv_pow2_of(hm);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          float4* p = reinterpret_cast<float4*>(hr + 8 * s);
          const float4 v = *p;
          *p = make_float4(dg * v.x, dg * v.y, dg * v.z, dg * v.w);
        }
        if (L.q == 0) {
          tks[8 * L.w + L.g] *= dg;
          dinv[8 * L.w + L.g] = 1.f / dg;
        }
      }
      __syncthreads();

      // ---- setup on the scaled channel (split TF32, as the TF32 kernel); a resident
      // factor slot holding the FP32 path's G'^{-T} replaces the Gram matrix and its
      // inversion
      int fl = 0;
      const float2* fin = nullptr;
      float2* fout = nullptr;
      if (A.fac) {
        if (A.opts & OPT_FAC_EXPORT)
          fout = A.fac + inst * (int64_t)fac_stride(KB);
        else if (A.fidx && A.fidx[inst] >= 0)
          fin = A.fac + A.fidx[inst];
      }
      const bool imported = fin && fin[KB * KB].x == 1.f;
      if (imported) {
        for (int idx = L.tid; idx < KB * KB; idx += NT) Es[idx] = fin[idx];
      } else {
#pragma unroll 1
        for (int ct = 0; ct < KW; ++ct) {  // G'^T rows 8w .. 8w + 7
          float e[4];
          S::template e_tile<true>(L, Hs, w, ct, e);
          float2* row = Es + (8 * L.w + L.g) * KB + 8 * ct + 2 * L.q;
          *reinterpret_cast<float4*>(row) = make_float4(e[0], e[2], e[1], e[3]);
        }
      }
      __syncthreads();
      if (K < KB && !imported) {  // padded users: unit Gram diagonal
        if (L.tid >= K && L.tid < KB) Es[L.tid * KB + L.tid] = make_float2(1.f, 0.f);
        __syncthreads();
      }
      bool singular = false, basis = false;
      const bool fast = imported || S::gj_fp32(L, Es, dsc, rowp, colp, A.cond_thr);
      if (fout) {
        for (int idx = L.tid; idx < KB * KB; idx += NT) fout[idx] = Es[idx];
        if (L.tid == 0) fout[KB * KB] = make_float2(fast ? 1.f : 0.f, 0.f);
      }
      if (!fast) {
        // FP64 path: the layers run split TF32 in an orthonormal basis of the
        // (scaled) channel's row space, S~^T in Es (S::basis_fp64)
        fl = S::basis_fp64(L, K, Hs, Es, gf, A64, reinterpret_cast<double*>(r64),
                           reinterpret_cast<double*>(c64), o64, tks);
        singular = (fl & PRECODE_F_SINGULAR) != 0;
        basis = !singular;
      }
      if (!singular) {
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
        S::update(L, Hs, ft, w);  // W^(0)' = S' G'^{-T} conj(H') (split TF32)
      }
      // with the basis, the global scale b scales W^(0)' and S~^T alike (below)
      // ---- the global scale b: max(|W^(0)'|, t') into [8, 16)
      float wm = fabsf(tks[L.lane % KB]);
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int k = 0; k < 4; ++k) wm = fmaxf(wm, fabsf(w[s][k]));
#pragma unroll
      for (int msk = 1; msk < 32; msk <<= 1) wm = fmaxf(wm, __shfl_xor_sync(FULL, wm, msk));
      if (L.lane == 0) wred[L.w] = wm;
      __syncthreads();
      wm = 0.f;
#pragma unroll
      for (int k = 0; k < KW; ++k) wm = fmaxf(wm, wred[k]);
      const float beta = 16.f * inv_pow2_of(wm);
#pragma unroll
      for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int k = 0; k < 4; ++k) w[s][k] *= beta;
      __syncthreads();  // every t', wred and raw-channel read done
      if (L.tid < KB) tks[L.tid] *= beta;
      if (basis)
        for (int idx = L.tid; idx < KB * KB; idx += NT) {
          const float2 v = Es[idx];
          Es[idx] = make_float2(beta * v.x, beta * v.y);
        }
      const bool tf32_layers = (fl & PRECODE_F_FP64_CHOL) != 0;
      if (!tf32_layers && !singular) to_chunks(L, Hs);
      __syncthreads();

      // ---- layers (scaled units)
      const int T = A.T;
      float rss = 0.f;
      if (!singular) {
#pragma unroll 1
        for (int l = 0; l < T; ++l) {
          S::shrink(L, np, fb, par, fmaxf(__ldg(A.step + l), 0.f) * beta, w);
          par ^= 1;
          if (tf32_layers) {
            S::residual_f(L, Hs, gf, tks, 1.f, w, ft, basis ? Es : nullptr);
            S::update(L, Hs, ft, w);
            continue;
          }
          const float xs = residual_fh(L, Hs, gf, tks, w, ft);
          if (xs == 1.f)
            update_c<false>(L, Hs, ft, 1.f, w);
          else if (xs > 0.f)
            update_c<true>(L, Hs, ft, xs, w);
          else
            update_c_tf32(L, Hs, ft, w);
        }
        if (A.resid) {
          if (basis) {  // against the channel itself, scaled per user again (H' = D H)
            __syncthreads();
            if (L.tid < KB) dsc[L.tid] = 1.f / dinv[L.tid];
            __syncthreads();
            S::reload_channel(L, K, A.H + h_off, Hs, dsc);
          }
          rss = tf32_layers ? residual_ssh<true>(L, Hs, tks, dinv, w)
                            : residual_ssh<false>(L, Hs, tks, dinv, w);
#pragma unroll
          for (int msk = 1; msk < 32; msk <<= 1) rss += __shfl_xor_sync(FULL, rss, msk);
        }
      } else {
#pragma unroll
        for (int s = 0; s < NS; ++s)
#pragma unroll
          for (int k = 0; k < 4; ++k) w[s][k] = 0.f;
        if (L.w == 0 && L.lane == 0)
          for (int k = 0; k < KB; ++k) rss += (tks[k] * dinv[k]) * (tks[k] * dinv[k]);
      }
      if (L.lane == 0) wred[L.w] = rss;

      // ---- objective, next copy, W write-back (original units)
      const float f_out = 1.f / beta;
      float r[NQ];
      S::colsum(L, np, par, w, r);
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
          *reinterpret_cast<float4*>(Wg + 8 * s) =
              make_float4(f_out * w[s][0], f_out * w[s][2], f_out * w[s][1], f_out * w[s][3]);
      }
      if (L.tid == 0) {
        float rs = 0.f;
        for (int k = 0; k < KW; ++k) rs += wred[k];
        o *= f_out;
        const float res = sqrtf(rs) * f_out;
        if (!(o < FLT_MAX) || !(res < FLT_MAX)) fl |= PRECODE_F_NONFINITE;
        if (A.obj) A.obj[inst] = o;
        if (A.resid) A.resid[inst] = res;
        if (A.flags) A.flags[inst] = fl;
      }
    }
  }
};

template <int KW, int MB, int MINB>
__global__ void __launch_bounds__(KW * 32, MINB) solve_tcwh_kernel(SolveArgs A) {
  SolveTCWH<KW, MB>::run(A);
}

}  // namespace precode
