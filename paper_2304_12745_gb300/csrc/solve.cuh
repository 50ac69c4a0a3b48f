// Persistent deep-unfolded precoder kernel (both layer maps), FP32 complex.
//
// One "instance group" of TPI = GK*GM threads owns one problem instance at a
// time and keeps it on chip for all T layers:
//   * H (and, for the projected layer, Q = G^{-T} H^*) in shared memory, loaded
//     by one bulk async copy per instance (TMA engine, completion on an mbarrier);
//   * W in registers: thread (a, b) owns users k = a + GK*u (u < KB/GK) and
//     antenna pairs p = b + GM*i (i < MB/(2 GM)), i.e. antennas 2p and 2p+1.
// Per layer the only cross-antenna reduction is E = W H^T - S (K x K): every
// thread sums its antennas' share, then the GM threads of one user row reduce
// it through a bank-swizzled shared buffer into the K x K matrix Es.  Column
// norms (per antenna, over users) reduce over the GK user rows with warp
// shuffles (plus shared memory when a group spans several warps).
//
// Paper layer (Sec. V, Eq. unfoldednet):    E = W H^T - S;  V = W - eta E H^*;
//                                           W = prox_{lam eta ||.||_{2,1}}(V);  W^(0) = H^*.
// Projected layer (constraint of Eq. optim1): X = prox_{mu ||.||_{2,1}}(W);
//                                           W = X - (X H^T - S) Q,  Q = G^{-T} H^*;
//                                           W^(0) = S Q (the ZF precoder).
// Q is computed once per instance from the equilibrated Gram factorisation
// D G D = L' diag(d) L'^H (D = diag(G)^{-1/2}, L' unit lower): FP32, or FP64 when
// a pivot fails or max(d)/min(d) exceeds the threshold.  A projected layer then
// costs the same two K x K x M contractions as a paper layer.
#pragma once

#include <cfloat>
#include <cstdint>
#include <type_traits>

#include "device.cuh"
#include "kernel_args.h"
#include "precode.h"

namespace precode {

constexpr int kModePGD = 0;
constexpr int kModeProj = 1;
constexpr uint64_t kCopyWaitNs = 1000000000ull;  // 1 s bound on one channel copy

// Limit of one channel-copy wait for this launch (the plan may shorten it).
__device__ __forceinline__ uint64_t copy_wait_ns(const SolveArgs& A) {
  return A.wait_ns ? A.wait_ns : kCopyWaitNs;
}

__host__ __device__ constexpr int align_up(int x, int a) { return (x + a - 1) / a * a; }

template <int MODE, int KB, int MB, int GK, int GM, int JC_, int NW, bool DB = false>
struct SolveCfg {
  static constexpr int TPI = GK * GM;            // threads per instance
  static constexpr int UPT = KB / GK;            // users per thread
  static constexpr int PPT = MB / (2 * GM);      // antenna pairs per thread
  static constexpr int NA = 2 * PPT;             // antennas per thread
  static constexpr int JC = JC_;                 // residual columns per reduction pass
  static constexpr int NJC = KB / JC;
  static constexpr int THREADS = NW * 32;
  static constexpr int GROUPS = THREADS / TPI;   // instances resident per block
  static constexpr int WPG = TPI >= 32 ? TPI / 32 : 1;
  static constexpr int LPW = TPI >= 32 ? 32 : TPI;  // lanes of a group inside one warp
  static constexpr int PF = 2 * UPT * JC;        // partial floats per thread per pass
  static constexpr int SEG = PF / GM;            // reduced floats per thread per pass
  // partial-buffer row stride: one extra segment (or 16 B) of padding makes the
  // segment writes and the column reads bank-conflict free without index math
  static constexpr int RS = PF + (SEG % 4 == 0 ? 4 : SEG);
  static_assert(KB % GK == 0 && MB % (2 * GM) == 0, "lane grid must tile the bucket");
  static_assert(KB % JC == 0, "reduction passes tile the residual columns");
  static_assert((GM & (GM - 1)) == 0 && GM <= 32 && (GK & (GK - 1)) == 0, "powers of two");
  static_assert(TPI <= 32 ? (32 % TPI == 0) : (TPI % 32 == 0), "groups tile warps");
  static_assert(THREADS % TPI == 0 && THREADS <= 1024, "block holds whole groups");
  static_assert(PF % GM == 0 && (SEG == 1 || SEG == 2 || SEG % 4 == 0), "segment size");
  static_assert(SEG < 4 || (2 * JC) % SEG == 0, "a 4-float segment stays inside one user row");
  static_assert(TPI >= KB, "one thread per Gram column");
  static_assert(TPI <= 32 || GROUPS <= 15, "one named barrier per group");
  static_assert(MODE == kModePGD || MB >= 5 * KB, "FP64 scratch lives in the Q area");
  // per-group shared memory (bytes)
  static constexpr int H_OFF = 0;
  static constexpr int H_BYTES = KB * MB * 8;             // one channel buffer
  static constexpr int NHB = DB ? 2 : 1;                  // channel buffers (DB: prefetch depth 2)
  static constexpr int Q_OFF = H_OFF + NHB * H_BYTES;
  static constexpr int Q_BYTES = MODE == kModeProj ? KB * MB * 8 : 0;
  static constexpr int RED_OFF = Q_OFF + Q_BYTES;
  static constexpr int RED_BYTES = align_up(TPI * RS * 4, 16);
  static constexpr int E_OFF = RED_OFF + RED_BYTES;
  static constexpr int E_BYTES = KB * KB * 8;
  static constexpr int ST_OFF = E_OFF + E_BYTES;  // S~^T of the FP64 path's orthonormal basis
  static constexpr int ST_BYTES = MODE == kModeProj ? KB * KB * 8 : 0;
  static constexpr int NRM_OFF = ST_OFF + ST_BYTES;
  static constexpr int NRM_BYTES = WPG > 1 ? WPG * GM * NA * 4 : 0;
  static constexpr int SC_OFF = NRM_OFF + NRM_BYTES;  // t[KB] dsc[KB] piv[KB] misc[8] wsum[WPG]
  static constexpr int SC_BYTES = align_up((3 * KB + 8 + WPG) * 4, 16);
  static constexpr int BAR_OFF = SC_OFF + SC_BYTES;
  static constexpr int GROUP_BYTES = align_up(BAR_OFF + 8 * NHB, 16);
  static constexpr int SMEM_BYTES = GROUPS * GROUP_BYTES;
  static_assert(RED_BYTES >= 2 * KB * KB * 8, "Gauss-Jordan buffers live in the reduction buffer");
  static_assert(MODE == kModePGD || RED_BYTES >= KB * KB * 16, "FP64 inverse in reduction buffer");
};

template <int MODE, int KB, int MB, int GK, int GM, int JC_, bool EXACT, int NW, bool SPLIT, bool DB>
struct SolveKernel {
  using C = SolveCfg<MODE, KB, MB, GK, GM, JC_, NW, DB>;
  // register form of complex W and partial sums: scalar pairs (SPLIT) or float2
  using CT = typename std::conditional<SPLIT, cf, float2>::type;
  static constexpr int TPI = C::TPI, UPT = C::UPT, PPT = C::PPT, NA = C::NA, JC = C::JC,
                       NJC = C::NJC, PF = C::PF, SEG = C::SEG, RS = C::RS, WPG = C::WPG,
                       LPW = C::LPW;

  struct Ctx {
    float2* Hs;
    float2* Qs;
    float* red;
    float2* Es;
    float* nrm;
    float* tks;
    float* dsc;
    float* piv;
    int* misc;
    float* wsum;
    uint64_t* bar;
    int g, a, b, lane, wig, gid;
    unsigned wmask;
    int K, M;
  };

  using WReg = CT[UPT][NA];
  using EReg = CT[UPT][JC];

  __device__ __forceinline__ static int Kd(const Ctx& c) { return EXACT ? KB : c.K; }
  __device__ __forceinline__ static int Md(const Ctx& c) { return EXACT ? MB : c.M; }
  __device__ __forceinline__ static int user(const Ctx& c, int u) { return c.a + GK * u; }
  __device__ __forceinline__ static int pair(const Ctx& c, int i) { return c.b + GM * i; }
  __device__ __forceinline__ static bool uok(const Ctx& c, int u) {
    return EXACT || user(c, u) < c.K;
  }
  __device__ __forceinline__ static bool pok(const Ctx& c, int i) {
    return EXACT || 2 * pair(c, i) < c.M;
  }

  __device__ __forceinline__ static void gsync(const Ctx& c) {
    if constexpr (TPI <= 32) {
      __syncwarp(c.wmask);
    } else {
      asm volatile("bar.sync %0, %1;" ::"r"(c.gid + 1), "r"(TPI) : "memory");
    }
  }

  // w <- rows k_u of X (shared [K][M]) restricted to this thread's antennas.
  __device__ __forceinline__ static void load_rows(const Ctx& c, WReg& w, const float2* X) {
    const int M = Md(c);
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        if (uok(c, u) && pok(c, i)) {
          const float4 v = *reinterpret_cast<const float4*>(X + user(c, u) * M + 2 * pair(c, i));
          w[u][2 * i] = mkc<CT>(v.x, v.y);
          w[u][2 * i + 1] = mkc<CT>(v.z, v.w);
        } else {
          w[u][2 * i] = mkc<CT>(0.f, 0.f);
          w[u][2 * i + 1] = mkc<CT>(0.f, 0.f);
        }
      }
  }

  // e[u][jj] = sum over own antennas m of w[u][m] * X[j][m], j = jc*JC + jj.
  // Pairs outer, residual columns inner: consecutive multiply-adds go to
  // different accumulators.
  __device__ __forceinline__ static void partials(const Ctx& c, const WReg& w, const float2* X,
                                                  int jc, EReg& e) {
    const int K = Kd(c), M = Md(c);
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int jj = 0; jj < JC; ++jj) e[u][jj] = mkc<CT>(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < PPT; ++i) {
      if (!pok(c, i)) continue;
#pragma unroll
      for (int jj = 0; jj < JC; ++jj) {
        const int j = jc * JC + jj;
        if (!EXACT && j >= K) continue;
        const float4 v = *reinterpret_cast<const float4*>(X + j * M + 2 * pair(c, i));
        const float2 x0 = make_float2(v.x, v.y), x1 = make_float2(v.z, v.w);
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          cmac(e[u][jj], w[u][2 * i], x0);
          cmac(e[u][jj], w[u][2 * i + 1], x1);
        }
      }
    }
  }

  __device__ __forceinline__ static float pf(const EReg& e, int f) {
    return (f & 1) ? e[f / (2 * JC)][(f >> 1) % JC].y : e[f / (2 * JC)][(f >> 1) % JC].x;
  }

  // S~^T [KB][KB] of an instance solved in the orthonormal basis (the buffer after E).
  __device__ __forceinline__ static float2* st_buf(const Ctx& c) {
    return reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(c.Es) + C::E_BYTES);
  }

  // Sum the partials of the GM threads of this user row; the reduced entries
  // (minus the target when SUB_S: S on the diagonal, or all of S~^T when the
  // instance runs in the orthonormal basis (BASIS); times `scale`) go to Es[k][j].
  // Returns the sum of squares of the entries this thread wrote.
  __device__ __forceinline__ static float reduce(const Ctx& c, const EReg& e, int jc,
                                                 float scale, bool sub_s, bool basis = false) {
    float* row = c.red + (c.a * GM + c.b) * RS;
#pragma unroll
    for (int s = 0; s < GM; ++s) {
      float* dst = row + s * SEG;
      if constexpr (SEG % 4 == 0) {
#pragma unroll
        for (int q = 0; q < SEG; q += 4)
          *reinterpret_cast<float4*>(dst + q) =
              make_float4(pf(e, s * SEG + q), pf(e, s * SEG + q + 1), pf(e, s * SEG + q + 2),
                          pf(e, s * SEG + q + 3));
      } else if constexpr (SEG == 2) {
        *reinterpret_cast<float2*>(dst) = make_float2(pf(e, s * SEG), pf(e, s * SEG + 1));
      } else {
        *dst = pf(e, s);
      }
    }
    __syncwarp(c.wmask);
    // gather the GM partial segments of this thread's slot, then sum them as a tree
    float part[GM][SEG];
#pragma unroll
    for (int bb = 0; bb < GM; ++bb) {
      const float* src = c.red + (c.a * GM + bb) * RS + c.b * SEG;
      if constexpr (SEG % 4 == 0) {
#pragma unroll
        for (int q = 0; q < SEG; q += 4) {
          const float4 v = *reinterpret_cast<const float4*>(src + q);
          part[bb][q] = v.x;
          part[bb][q + 1] = v.y;
          part[bb][q + 2] = v.z;
          part[bb][q + 3] = v.w;
        }
      } else if constexpr (SEG == 2) {
        const float2 v = *reinterpret_cast<const float2*>(src);
        part[bb][0] = v.x;
        part[bb][1] = v.y;
      } else {
        part[bb][0] = *src;
      }
    }
#pragma unroll
    for (int span = 1; span < GM; span <<= 1)
#pragma unroll
      for (int bb = 0; bb + span < GM; bb += 2 * span)
#pragma unroll
        for (int q = 0; q < SEG; ++q) part[bb][q] += part[bb + span][q];
    float acc[SEG];
#pragma unroll
    for (int q = 0; q < SEG; ++q) acc[q] = part[0][q];
    float ssq = 0.f;
    float* Ef = reinterpret_cast<float*>(c.Es);
#pragma unroll
    for (int q = 0; q < SEG; ++q) {
      const int f = c.b * SEG + q;
      const int u = f / (2 * JC);
      const int jj = (f >> 1) % JC;
      const int k = user(c, u);
      const int j = jc * JC + jj;
      float v = acc[q];
      if (basis) {
        v -= reinterpret_cast<const float*>(st_buf(c))[(k * KB + j) * 2 + (f & 1)];
      } else if (sub_s && (f & 1) == 0 && j == k && k < Kd(c)) {
        v -= c.tks[k];
      }
      v *= scale;
      ssq = fmaf(v, v, ssq);
      acc[q] = v;
      if constexpr (SEG < 4) Ef[(k * KB + j) * 2 + (f & 1)] = v;
    }
    if constexpr (SEG % 4 == 0) {
#pragma unroll
      for (int q = 0; q < SEG; q += 4) {
        const int f = c.b * SEG + q;
        const int k = user(c, f / (2 * JC));
        const int j = jc * JC + ((f >> 1) % JC);
        *reinterpret_cast<float4*>(Ef + (k * KB + j) * 2) =
            make_float4(acc[q], acc[q + 1], acc[q + 2], acc[q + 3]);
      }
    }
    __syncwarp(c.wmask);
    return ssq;
  }

  // Squared column norms over all users, identical in every thread of a column.
  __device__ __forceinline__ static void colnorm2(const Ctx& c, const WReg& w, float (&r2)[NA]) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      float s = 0.f;
#pragma unroll
      for (int u = 0; u < UPT; ++u) s = fmaf(w[u][q].x, w[u][q].x, fmaf(w[u][q].y, w[u][q].y, s));
      r2[q] = s;
    }
#pragma unroll
    for (int msk = GM; msk < LPW; msk <<= 1)
#pragma unroll
      for (int q = 0; q < NA; ++q) r2[q] += __shfl_xor_sync(c.wmask, r2[q], msk);
    if constexpr (WPG > 1) {
      float* buf = c.nrm;
      if (c.lane < GM)
#pragma unroll
        for (int q = 0; q < NA; ++q) buf[(c.wig * GM + c.b) * NA + q] = r2[q];
      gsync(c);
#pragma unroll
      for (int q = 0; q < NA; ++q) {
        float s = 0.f;
        for (int ww = 0; ww < WPG; ++ww) s += buf[(ww * GM + c.b) * NA + q];
        r2[q] = s;
      }
      gsync(c);  // buffer free for the next call
    }
  }

  // Group soft threshold per antenna column: w_m <- max(0, 1 - tau/||w_m||) w_m.
  __device__ __forceinline__ static void shrink(WReg& w, const float (&r2)[NA], float tau) {
    const float tau2 = tau * tau;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const float s = (r2[q] > tau2) ? (1.f - tau * rsqrtf(r2[q])) : 0.f;
#pragma unroll
      for (int u = 0; u < UPT; ++u) {
        w[u][q].x *= s;
        w[u][q].y *= s;
      }
    }
  }

  // w -= Es[k_u][:] * X  (CJ: X conjugated), X shared [K][M].
  template <bool CJ>
  __device__ __forceinline__ static void update(const Ctx& c, WReg& w, const float2* X) {
    const int K = Kd(c), M = Md(c);
#pragma unroll 4
    for (int j = 0; j < KB; ++j) {
      if (!EXACT && j >= K) break;
      {
        float2 ej[UPT];
#pragma unroll
        for (int u = 0; u < UPT; ++u) ej[u] = c.Es[user(c, u) * KB + j];
        const float2* row = X + j * M;
#pragma unroll
        for (int i = 0; i < PPT; ++i) {
          if (!pok(c, i)) continue;
          const float4 v = *reinterpret_cast<const float4*>(row + 2 * pair(c, i));
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
  }

  // Projected-layer setup from Es = G^T = conj(H H^H) (Hermitian, same diagonal
  // and conditioning as G).  Its inverse is G^{-T}, so Q = G^{-T} H^* is formed
  // directly.  The equilibrated matrix D G^T D (D = diag(G)^{-1/2}) is inverted
  // in place by Gauss-Jordan elimination without pivoting, every thread owning
  // fixed entries; its pivots are the LDL^H pivots d_p, so max(d)/min(d) is the
  // condition estimate that decides the FP64 fallback.  Writes Q to Qs and
  // W^(0) = S Q into w.  Returns the instance flags.  On the FP64 path the layers
  // run in an orthonormal basis of the channel's row space with BASIS
  // (setup_proj_fp64_basis), else through Q formed in FP64 (setup_proj_fp64).
  template <bool BASIS = false>
  __device__ static int setup_proj(Ctx& c, WReg& w, float cond_thr) {
    const int K = Kd(c), M = Md(c);
    constexpr int NE = (KB * KB + TPI - 1) / TPI;  // matrix entries per thread
    constexpr int LKB = KB == 4 ? 2 : KB == 8 ? 3 : KB == 16 ? 4 : 5;
    static_assert((1 << LKB) == KB, "bucket K is a power of two");
    if (c.g < K) c.dsc[c.g] = rsqrtf(c.Es[c.g * KB + c.g].x);
    gsync(c);
    // A0 = D G^T D in the reduction buffer (two K x K buffers ping-pong there)
    float2* A0 = reinterpret_cast<float2*>(c.red);
    float2* A1 = A0 + KB * KB;
#pragma unroll
    for (int r = 0; r < NE; ++r) {
      const int idx = c.g + r * TPI;
      const int i = idx >> LKB, j = idx & (KB - 1);
      if (idx < KB * KB && i < K && j < K) {
        const float s = c.dsc[i] * c.dsc[j];
        const float2 v = c.Es[i * KB + j];
        A0[i * KB + j] = make_float2(v.x * s, v.y * s);
      }
    }
    gsync(c);
    bool fail = false;
    float dmin = FLT_MAX, dmax = 0.f;
    float2* cur = A0;
    float2* nxt = A1;
    for (int p = 0; p < K; ++p) {
      const float d = cur[p * KB + p].x;
      if (!(d > 0.f) || !(d < FLT_MAX)) {
        fail = true;
        break;
      }
      dmin = fminf(dmin, d);
      dmax = fmaxf(dmax, d);
      const float inv = 1.f / d;
#pragma unroll
      for (int r = 0; r < NE; ++r) {
        const int idx = c.g + r * TPI;
        const int i = idx >> LKB, j = idx & (KB - 1);
        if (idx < KB * KB && i < K && j < K) {
          float2 v;
          if (i == p && j == p) {
            v = make_float2(inv, 0.f);
          } else if (i == p) {
            const float2 a = cur[p * KB + j];
            v = make_float2(a.x * inv, a.y * inv);
          } else if (j == p) {
            const float2 a = cur[i * KB + p];
            v = make_float2(-a.x * inv, -a.y * inv);
          } else {
            const float2 aip = cur[i * KB + p], apj = cur[p * KB + j];
            v = cur[i * KB + j];
            cmsub(v, make_float2(aip.x * inv, aip.y * inv), apj);
          }
          nxt[i * KB + j] = v;
        }
      }
      gsync(c);
      float2* tmp = cur;
      cur = nxt;
      nxt = tmp;
    }
    if (fail || dmax > cond_thr * dmin)
      return BASIS ? setup_proj_fp64_basis(c, w) : setup_proj_fp64(c, w);
    // G^{-T} = D (D G^T D)^{-1} D  -> Es
#pragma unroll
    for (int r = 0; r < NE; ++r) {
      const int idx = c.g + r * TPI;
      const int i = idx >> LKB, j = idx & (KB - 1);
      if (idx < KB * KB && i < K && j < K) {
        const float s = c.dsc[i] * c.dsc[j];
        const float2 v = cur[i * KB + j];
        c.Es[i * KB + j] = make_float2(v.x * s, v.y * s);
      }
    }
    gsync(c);
    // Q = G^{-T} H^* on own entries; W^(0) = t_k Q
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int q = 0; q < NA; ++q) w[u][q] = mkc<CT>(0.f, 0.f);
    for (int l = 0; l < K; ++l) {
      float2 gl[UPT];
#pragma unroll
      for (int u = 0; u < UPT; ++u) gl[u] = c.Es[user(c, u) * KB + l];
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        if (!pok(c, i)) continue;
        const float4 v = *reinterpret_cast<const float4*>(c.Hs + l * M + 2 * pair(c, i));
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          cmac_conj(w[u][2 * i], gl[u], make_float2(v.x, v.y));
          cmac_conj(w[u][2 * i + 1], gl[u], make_float2(v.z, v.w));
        }
      }
    }
    store_q_and_start(c, w);
    return 0;
  }

  // Q = w into Qs for own entries, then w <- t_k Q.
  __device__ __forceinline__ static void store_q_and_start(Ctx& c, WReg& w) {
    const int M = Md(c);
#pragma unroll
    for (int u = 0; u < UPT; ++u) {
      const float tk = uok(c, u) ? c.tks[user(c, u)] : 0.f;
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        const CT q0 = w[u][2 * i];
        const CT q1 = w[u][2 * i + 1];
        if (uok(c, u) && pok(c, i))
          *reinterpret_cast<float4*>(c.Qs + user(c, u) * M + 2 * pair(c, i)) =
              make_float4(q0.x, q0.y, q1.x, q1.y);
        w[u][2 * i] = mkc<CT>(tk * q0.x, tk * q0.y);
        w[u][2 * i + 1] = mkc<CT>(tk * q1.x, tk * q1.y);
      }
    }
    gsync(c);
  }

  // FP64 Gram matrix of the channel rows and its LDL^H factorisation (no
  // equilibration; a pivot below 1e-12 times its Gram diagonal entry means
  // rank(H) < K), in the FP64 scratch of the Q area: G[i][j] (j < i) holds
  // L[i][j] d_j, pv[i] = 1 / d_i.  Returns the instance flags.
  __device__ static int fp64_ldl(Ctx& c) {
    const int K = Kd(c), M = Md(c);
    double2* G = reinterpret_cast<double2*>(c.Qs);
    double* orig = reinterpret_cast<double*>(G + 2 * KB * KB);
    double* pv = orig + KB;
    for (int idx = c.g; idx < K * K; idx += TPI) {
      const int i = idx / K, j = idx - i * K;
      if (j > i) continue;
      double sr = 0.0, si = 0.0;
      for (int m = 0; m < M; ++m) {
        const float2 x = c.Hs[i * M + m], y = c.Hs[j * M + m];
        sr += (double)x.x * y.x + (double)x.y * y.y;
        si += (double)x.y * y.x - (double)x.x * y.y;
      }
      G[i * KB + j] = make_double2(sr, si);
    }
    gsync(c);
    if (c.g < K) orig[c.g] = G[c.g * KB + c.g].x;
    gsync(c);
    int fl = PRECODE_F_FP64_CHOL;
    bool singular = false;
    for (int j = 0; j < K; ++j) {
      const double d = G[j * KB + j].x;
      if (!(d > 1e-12 * orig[j]) || !(d < DBL_MAX)) {
        singular = true;
        if (!(orig[j] < DBL_MAX) || orig[j] != orig[j]) fl |= PRECODE_F_NONFINITE;
        break;
      }
      const double inv = 1.0 / d;
      const int R = K - 1 - j;
      for (int idx = c.g; idx < R * R; idx += TPI) {
        const int i = j + 1 + idx / R, l = j + 1 + idx % R;
        if (l > i) continue;
        const double2 aij = G[i * KB + j], alj = G[l * KB + j];
        const double ar = aij.x * inv, ai = aij.y * inv;
        double2 v = G[i * KB + l];
        v.x -= ar * alj.x + ai * alj.y;  // a * conj(b)
        v.y -= ai * alj.x - ar * alj.y;
        G[i * KB + l] = v;
      }
      gsync(c);
    }
    if (singular) {
      gsync(c);
      return fl | PRECODE_F_SINGULAR;
    }
    if (c.g < K) pv[c.g] = 1.0 / G[c.g * KB + c.g].x;
    gsync(c);
    return fl;
  }

  // Li = L^{-1} (unit lower triangular, row stride KB) from fp64_ldl's factors.
  __device__ static void fp64_linv(Ctx& c, double2* Li) {
    const int K = Kd(c);
    const double2* G = reinterpret_cast<const double2*>(c.Qs);
    const double* pv = reinterpret_cast<const double*>(G + 2 * KB * KB) + KB;
    if (c.g < K) {
      const int col = c.g;
      Li[col * KB + col] = make_double2(1.0, 0.0);
      for (int i = col + 1; i < K; ++i) {
        double sr = 0.0, si = 0.0;
        for (int p = col; p < i; ++p) {
          const double2 a = G[i * KB + p], x = Li[p * KB + col];
          const double ar = a.x * pv[p], ai = a.y * pv[p];
          sr += ar * x.x - ai * x.y;
          si += ar * x.y + ai * x.x;
        }
        Li[i * KB + col] = make_double2(-sr, -si);
      }
    }
    gsync(c);
  }

  // FP64 Gram, LDL^H and inverse.  G^{-1} goes to the reduction buffer (double2,
  // K x K with row stride KB) unless the flags say singular.
  __device__ static int fp64_inverse(Ctx& c) {
    const int K = Kd(c);
    const int fl = fp64_ldl(c);
    if (fl & PRECODE_F_SINGULAR) return fl;
    double2* G = reinterpret_cast<double2*>(c.Qs);
    double2* U = G + KB * KB;
    const double* pv = reinterpret_cast<const double*>(G + 2 * KB * KB) + KB;
    double2* Gi = reinterpret_cast<double2*>(c.red);
    fp64_linv(c, U);
    for (int idx = c.g; idx < K * K; idx += TPI) {
      const int i = idx / K, j = idx - i * K;
      double sr = 0.0, si = 0.0;
      for (int p = (i > j ? i : j); p < K; ++p) {
        const double2 upi = U[p * KB + i], upj = U[p * KB + j];
        // conj(U_pi) U_pj / d_p
        sr += (upi.x * upj.x + upi.y * upj.y) * pv[p];
        si += (upi.x * upj.y - upi.y * upj.x) * pv[p];
      }
      Gi[i * KB + j] = make_double2(sr, si);
    }
    gsync(c);
    return fl;
  }

  // FP64 Gram factorisation and an orthonormal basis of the channel's row space.
  // With G = H H^H = L D L^H (FP64) the rows of
  //   U = D^{-1/2} L^{-1} H      (K x M, U U^H = I)
  // span the same space as H's, and H W^T = S becomes U W^T = S~ with the lower
  // triangular S~ = D^{-1/2} L^{-1} S.  The projection onto that set is
  //   P(X) = X - (X U^T - S~^T) conj(U),
  // the same map as X - (X H^T - S) G^{-T} H^*, but rounding U to FP32 perturbs
  // an orthogonal projector by O(u) whatever the conditioning of H, whereas
  // Q = G^{-T} H^* in FP32 carries O(u sqrt(cond G)) into every layer and the
  // residual's cancellation error is amplified by 1 / sigma_min(H).  Writes U
  // over the channel in Hs, conj(U) into Qs and S~^T ([KB][KB], zero outside
  // K x K) into St, all from FP64 sums rounded once; L^{-1} uses the reduction
  // buffer and d^{-1/2} the E buffer.  Returns the instance flags (FP64_CHOL,
  // plus SINGULAR / NONFINITE, in which case nothing is written).
  __device__ static int fp64_basis(Ctx& c, float2* St) {
    const int K = Kd(c), M = Md(c);
    const int fl = fp64_ldl(c);
    if (fl & PRECODE_F_SINGULAR) return fl;
    double2* Li = reinterpret_cast<double2*>(c.red);
    fp64_linv(c, Li);
    double* isd = reinterpret_cast<double*>(c.Es);  // d_i^{-1/2}
    {
      const double* pv = reinterpret_cast<const double*>(reinterpret_cast<double2*>(c.Qs) + 2 * KB * KB) + KB;
      if (c.g < K) isd[c.g] = sqrt(pv[c.g]);
    }
    gsync(c);  // the FP64 scratch in the Q area is read out
    for (int idx = c.g; idx < K * M; idx += TPI) {
      const int i = idx / M, m = idx - i * M;
      double ur = 0.0, ui = 0.0;
      for (int p = 0; p <= i; ++p) {
        const double2 l = Li[i * KB + p];
        const float2 h = c.Hs[p * M + m];
        ur += l.x * h.x - l.y * h.y;
        ui += l.x * h.y + l.y * h.x;
      }
      c.Qs[idx] = make_float2((float)(ur * isd[i]), (float)(-ui * isd[i]));  // conj(U)
    }
    for (int idx = c.g; idx < KB * KB; idx += TPI) {
      const int k = idx / KB, j = idx - k * KB;
      float2 v = make_float2(0.f, 0.f);
      if (k < K && j < K && k <= j) {  // S~^T[k][j] = S~[j][k] = d_j^{-1/2} Li[j][k] t_k
        const double2 l = Li[j * KB + k];
        const double sc = isd[j] * (double)c.tks[k];
        v = make_float2((float)(l.x * sc), (float)(l.y * sc));
      }
      St[idx] = v;
    }
    gsync(c);  // U complete: it replaces the channel
    for (int idx = c.g; idx < K * M; idx += TPI) {
      const float2 q = c.Qs[idx];
      c.Hs[idx] = make_float2(q.x, -q.y);
    }
    gsync(c);
    return fl;
  }

  // FP64 path of the projected-layer setup in the orthonormal basis (fp64_basis):
  // S~^T into st_buf, misc[2] set (the layers subtract S~^T and the final residual
  // reads the channel again) and W^(0) = S~^T conj(U) (the ZF precoder) into w.
  // Returns the instance flags.
  __device__ static int setup_proj_fp64_basis(Ctx& c, WReg& w) {
    const int K = Kd(c), M = Md(c);
    float2* const St = st_buf(c);
    const int fl = fp64_basis(c, St);
    if (fl & PRECODE_F_SINGULAR) {
#pragma unroll
      for (int u = 0; u < UPT; ++u)
#pragma unroll
        for (int q = 0; q < NA; ++q) w[u][q] = mkc<CT>(0.f, 0.f);
      return fl;
    }
    // W^(0) = S~^T conj(U) on own entries (the rows of U are orthonormal: no
    // cancellation in these sums)
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int q = 0; q < NA; ++q) w[u][q] = mkc<CT>(0.f, 0.f);
    for (int j = 0; j < K; ++j) {
      float2 sj[UPT];
#pragma unroll
      for (int u = 0; u < UPT; ++u) sj[u] = St[user(c, u) * KB + j];
#pragma unroll
      for (int i = 0; i < PPT; ++i) {
        if (!pok(c, i)) continue;
        const float4 v = *reinterpret_cast<const float4*>(c.Qs + j * M + 2 * pair(c, i));
#pragma unroll
        for (int u = 0; u < UPT; ++u) {
          cmac(w[u][2 * i], sj[u], make_float2(v.x, v.y));
          cmac(w[u][2 * i + 1], sj[u], make_float2(v.z, v.w));
        }
      }
    }
    if (c.g == 0) c.misc[2] = 1;
    gsync(c);
    return fl;
  }

  // FP64 path of the projected-layer setup: fp64_inverse, then Q =
  // conj(G^{-1} H) on own entries in FP64, rounded once, into Qs and W^(0) = S Q
  // into w (zero when singular).  Returns the instance flags.
  __device__ static int setup_proj_fp64(Ctx& c, WReg& w) {
    const int K = Kd(c), M = Md(c);
    const int fl = fp64_inverse(c);
    if (fl & PRECODE_F_SINGULAR) {
#pragma unroll
      for (int u = 0; u < UPT; ++u)
#pragma unroll
        for (int q = 0; q < NA; ++q) w[u][q] = mkc<CT>(0.f, 0.f);
      return fl;
    }
    const double2* Gi = reinterpret_cast<const double2*>(c.red);
    // own entries of conj(G^{-1} H) in FP64, rounded once
#pragma unroll
    for (int u = 0; u < UPT; ++u)
#pragma unroll
      for (int i = 0; i < PPT; ++i)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          double zr = 0.0, zi = 0.0;
          if (uok(c, u) && pok(c, i)) {
            const int k = user(c, u), m = 2 * pair(c, i) + h;
            for (int l = 0; l < K; ++l) {
              const double2 gkl = Gi[k * KB + l];
              const float2 x = c.Hs[l * M + m];
              zr += gkl.x * x.x - gkl.y * x.y;
              zi += gkl.x * x.y + gkl.y * x.x;
            }
          }
          w[u][2 * i + h] = mkc<CT>((float)zr, (float)-zi);  // Q = conj(G^{-1} H)
        }
    gsync(c);  // every thread is done with the FP64 scratch before Q overwrites it
    store_q_and_start(c, w);
    return fl;
  }

  // Paper-layer per-instance step normalisation 1 / max_k sum_j |G_kj|, from
  // Es = G^T (the row sums of |G^T| and |G| agree).
  __device__ static float inv_gershgorin(Ctx& c) {
    const int K = Kd(c);
    if (c.g < K) {
      float s = 0.f;
      for (int j = 0; j < K; ++j) {
        const float2 v = c.Es[c.g * KB + j];
        s += sqrtf(v.x * v.x + v.y * v.y);
      }
      c.dsc[c.g] = s;
    }
    gsync(c);
    float L = 0.f;
    for (int k = 0; k < K; ++k) L = fmaxf(L, c.dsc[k]);
    gsync(c);
    return 1.f / L;
  }

  __device__ static void run(const SolveArgs& A) {
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
    unsigned char* gs = smem + c.gid * C::GROUP_BYTES;
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
    c.Hs = reinterpret_cast<float2*>(gs + C::H_OFF);

    constexpr int NHB = C::NHB;
    if (c.g == 0)
      for (int q = 0; q < NHB; ++q) mbar_init(c.bar + q, 1);
    fence_mbar_init();
    __syncthreads();

    float2* const hbuf0 = reinterpret_cast<float2*>(gs + C::H_OFF);
    uint32_t phases = 0;  // bit q: parity of the next completion of buffer q
    const int64_t n_inst = A.tbl ? (int64_t)(*A.count) : A.B;
    const int64_t stride = (int64_t)gridDim.x * C::GROUPS;
    // where instance `it` lives: H / W / t offsets and shape
    auto locate = [&](int64_t it, int64_t& inst, int64_t& h_off, int64_t& w_off, int64_t& t_off,
                      int& Kr, int& Mr) {
      if (A.tbl) {
        inst = A.index[it];
        const InstDesc d = A.tbl[inst];
        h_off = d.h_off;
        w_off = d.w_off;
        t_off = d.t_off;
        Kr = d.K;
        Mr = d.M;
      } else {
        inst = it;
        Kr = A.K;
        Mr = A.M;
        h_off = it * (int64_t)A.K * A.M;
        w_off = h_off;
        t_off = it * A.t_stride;
      }
    };
    // one bulk async copy of instance `it`'s channel into channel buffer q
    auto issue_copy = [&](int64_t it, int q) {
      if (c.g != 0 || it >= n_inst || (A.opts & OPT_STALL_COPY)) return;
      int64_t inst, h_off, w_off, t_off;
      int Kr, Mr;
      locate(it, inst, h_off, w_off, t_off, Kr, Mr);
      const uint32_t bytes = (uint32_t)((EXACT ? KB : Kr) * (EXACT ? MB : Mr)) * 8u;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(c.bar + q, bytes);
      bulk_g2s(hbuf0 + q * (KB * MB), A.H + h_off, bytes, c.bar + q);
    };
    WReg w;
    EReg e;
    float r2[NA];
    const int64_t first = (int64_t)blockIdx.x * C::GROUPS + c.gid;
    for (int q = 0; q < NHB; ++q) issue_copy(first + q * stride, q);
    int cur = 0;  // channel buffer of the current instance
#pragma unroll 1
    for (int64_t it = first; it < n_inst; it += stride, cur = (cur + 1) % NHB) {
      int64_t inst, h_off, w_off, t_off;
      locate(it, inst, h_off, w_off, t_off, c.K, c.M);
      const int K = Kd(c), M = Md(c);
      c.Hs = hbuf0 + cur * (KB * MB);
      const uint32_t par = (phases >> cur) & 1u;

      // ---- wait for this instance's channel (its copy was issued earlier)
      gsync(c);  // every thread of the group is done with the previous instance
      if (c.g < K) c.tks[c.g] = A.t[t_off + c.g];
      if (c.g == 0) c.misc[2] = 0;  // not (yet) in the orthonormal basis
      if (c.g == 0) c.misc[0] = mbar_wait_bounded(c.bar + cur, par, copy_wait_ns(A)) ? 1 : 0;
      gsync(c);
      if (c.misc[0] == 0) {
        // the copy did not land in time: report, then wait (bounded) for it
        // before this group's buffers can be reused; give up the group if not.
        if (c.g == 0) {
          atomicAdd(A.err, 1ull);
          if (A.flags) A.flags[inst] = PRECODE_F_TIMEOUT;
          c.misc[1] = mbar_wait_bounded(c.bar + cur, par, copy_wait_ns(A)) ? 1 : 0;
        }
        gsync(c);
        if (c.misc[1] == 0) return;
        phases ^= 1u << cur;
        issue_copy(it + NHB * stride, cur);
        continue;
      }
      if (c.g != 0) mbar_wait_bounded(c.bar + cur, par, copy_wait_ns(A));  // already complete
      phases ^= 1u << cur;

      // ---- steps -1 .. T of one instance.  Step -1 (Gram, when needed) and
      // step T (final residual, when requested) share the residual code of the
      // layers, so its unrolled body exists once in the kernel.
      int fl = 0;
      const int T = A.T;
      const bool need_gram = (MODE == kModeProj) || (A.opts & OPT_STEP_NORMALISED);
      const int last = A.resid ? T : T - 1;
      float invL = 1.f, rs = 0.f;
      load_rows(c, w, c.Hs);
#pragma unroll
      for (int u = 0; u < UPT; ++u)
#pragma unroll
        for (int q = 0; q < NA; ++q) w[u][q].y = -w[u][q].y;  // conj(H) rows
#pragma unroll 1
      for (int s = need_gram ? -1 : 0; s <= last; ++s) {
        float scale = 1.f;
        if (s >= 0 && s < T) {
          if constexpr (MODE == kModeProj) {
            colnorm2(c, w, r2);
            shrink(w, r2, fmaxf(__ldg(A.step + s), 0.f));
          } else {
            scale = __ldg(A.step + s) * invL;
          }
        }
        rs = 0.f;
        // the final residual of an instance solved in the orthonormal basis is
        // taken against the channel itself, read again from global memory
        const float2* X = c.Hs;
        bool basis = false;
        if constexpr (MODE == kModeProj) {
          if (c.misc[2]) {
            if (s == T) {
              int64_t i0, ho, wo, to;
              int k0, m0;
              locate(it, i0, ho, wo, to, k0, m0);
              X = A.H + ho;
            } else {
              basis = true;
            }
          }
        }
#pragma unroll 1
        for (int jc = 0; jc < NJC; ++jc) {
          partials(c, w, X, jc, e);
          rs += reduce(c, e, jc, scale, s >= 0, basis);
        }
        if (s < 0) {
          // Es = sum_m conj(H_km) H_jm = G^T
          gsync(c);
          if constexpr (MODE == kModeProj) {
            fl = setup_proj<true>(c, w, A.cond_thr);
            if (fl & PRECODE_F_SINGULAR) break;
          } else {
            invL = inv_gershgorin(c);  // w still holds W^(0) = H^*
          }
          continue;
        }
        if (s == T) break;  // final residual only
        if constexpr (MODE == kModeProj) {
          update<false>(c, w, c.Qs);
        } else {
          update<true>(c, w, c.Hs);
          colnorm2(c, w, r2);
          shrink(w, r2, fmaxf(fmaxf(__ldg(A.lam + s), 0.f) * scale, 0.f));
        }
      }
      if (fl & PRECODE_F_SINGULAR) {
        // W = 0: objective 0, residual ||S||_F
        rs = 0.f;
        if (c.g == 0)
          for (int k = 0; k < K; ++k) rs += c.tks[k] * c.tks[k];
      }

      // ---- the channel buffer is free: start the next instance's copy, then
      // finish this one (objective, residual, W) while it is in flight
      gsync(c);
      issue_copy(it + NHB * stride, cur);
      colnorm2(c, w, r2);
      float o = 0.f;
#pragma unroll
      for (int q = 0; q < NA; ++q) o += sqrtf(r2[q]);
#pragma unroll
      for (int msk = 1; msk < GM; msk <<= 1) o += __shfl_xor_sync(c.wmask, o, msk);
      if (A.resid && !(fl & PRECODE_F_SINGULAR)) {
#pragma unroll
        for (int msk = 1; msk < LPW; msk <<= 1) rs += __shfl_xor_sync(c.wmask, rs, msk);
        if constexpr (WPG > 1) {
          if (c.lane == 0) c.wsum[c.wig] = rs;
          gsync(c);
          rs = 0.f;
          for (int ww = 0; ww < WPG; ++ww) rs += c.wsum[ww];
        }
      }
#pragma unroll
      for (int u = 0; u < UPT; ++u)
#pragma unroll
        for (int i = 0; i < PPT; ++i)
          if (uok(c, u) && pok(c, i))
            *reinterpret_cast<float4*>(A.W + w_off + (int64_t)user(c, u) * M + 2 * pair(c, i)) =
                make_float4(w[u][2 * i].x, w[u][2 * i].y, w[u][2 * i + 1].x, w[u][2 * i + 1].y);
      if (c.g == 0) {
        if (!(o < FLT_MAX) || !(rs < FLT_MAX)) fl |= PRECODE_F_NONFINITE;
        if (A.obj) A.obj[inst] = o;
        if (A.resid) A.resid[inst] = sqrtf(rs);
        if (A.flags) A.flags[inst] = fl;
      }
    }
  }
};

template <int MODE, int KB, int MB, int GK, int GM, int JC, bool EXACT, int NW, int MINB,
          bool SPLIT, bool DB>
__global__ void __launch_bounds__(NW * 32, MINB) solve_kernel(SolveArgs A) {
  SolveKernel<MODE, KB, MB, GK, GM, JC, EXACT, NW, SPLIT, DB>::run(A);
}

}  // namespace precode
