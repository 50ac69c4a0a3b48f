// Uneven-batch solve that allocates nothing.
//
// Some callers cannot allocate device memory on their fast path: a real-time
// baseband / L1 processing loop that reserves all of its memory at start-up and
// must never block on the allocator (cudaMalloc can synchronise the device and
// take milliseconds), or a component that lives inside a host application
// whose memory manager owns every device byte.  For them this file offers
// precode_solve_varlen_static: the same bucketed solve as precode_solve_varlen,
// without a plan object, whose scratch (per-bucket instance lists, bucket
// counters, the device wait-timeout counter) is one file-scope __device__
// array of fixed size.  Every GPU that loads this library holds that array
// until the process exits.
//
// The array's name in host code is only a host-side stand-in, not a device
// address, so the first call on each device (with that device current) asks
// the runtime for the real address with cudaGetSymbolAddress and caches it.
// That first call should therefore come before any stream capture.  All calls
// share the array and a call leaves its contents behind: the counters are
// cleared at the start of every call, and calls whose work overlaps on the GPU
// race on the array.
#include <cuda_runtime.h>

#include <mutex>

#include "api_internal.h"

namespace precode {

namespace {

constexpr int64_t kMaxInst = PRECODE_STATIC_MAX_INSTANCES;
constexpr int kMaxBk = PRECODE_STATIC_MAX_BUCKETS;
// layout (int32 words): [kMaxBk][kMaxInst] instance lists | kMaxBk counters |
// padding to 8 bytes | one 64-bit wait-timeout counter
constexpr int64_t kCountOff = (int64_t)kMaxBk * kMaxInst;
constexpr int64_t kErrOff = kCountOff + kMaxBk + ((kCountOff + kMaxBk) & 1);
constexpr int64_t kWords = kErrOff + 2;

static __device__ __align__(256) int32_t g_varlen_scratch[kWords];

struct StaticBuckets {
  int n;
  int mode;
  int M[kMaxBk], K[kMaxBk], KB[kMaxBk], MB[kMaxBk], exact[kMaxBk];
};

// Same assignment rule as the plan-based path: an exact bucket of the shape,
// else the smallest generic bucket that holds it; rejected descriptors are
// flagged.  The lists and counters live in the static scratch.
__global__ void bucketize_static_kernel(const InstDesc* __restrict__ tbl, int64_t B,
                                        StaticBuckets bt, int32_t* __restrict__ scratch,
                                        int32_t* __restrict__ flags) {
  int32_t* count = scratch + kCountOff;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
       b += (int64_t)gridDim.x * blockDim.x) {
    const InstDesc d = tbl[b];
    const bool ok = d.K >= 1 && d.K <= PRECODE_MAX_K && d.M >= 2 && d.M <= PRECODE_MAX_M &&
                    (d.M & 1) == 0 && (bt.mode != PRECODE_LAYER_PROJ || d.K <= d.M) &&
                    d.h_off >= 0 && d.w_off >= 0 && d.t_off >= 0 && (d.h_off & 1) == 0 &&
                    (d.w_off & 1) == 0;
    int s = -1;
    if (ok) {
      for (int i = 0; i < bt.n; ++i)
        if (bt.exact[i] && bt.M[i] == d.M && bt.K[i] == d.K) s = i;
      if (s < 0) {
        int best = 1 << 30;
        for (int i = 0; i < bt.n; ++i)
          if (!bt.exact[i] && bt.KB[i] >= d.K && bt.MB[i] >= d.M && bt.KB[i] * bt.MB[i] < best) {
            best = bt.KB[i] * bt.MB[i];
            s = i;
          }
      }
    }
    if (s < 0) {
      if (flags) flags[b] = PRECODE_F_INVALID;
      continue;
    }
    const int pos = atomicAdd(count + s, 1);
    scratch[s * kMaxInst + pos] = (int32_t)b;
  }
}

// Per-device address of the scratch array (set up on the first call on a device).
std::mutex g_setup_mu;
int32_t* g_scratch_ptr[64] = {};

precode_status_t scratch_address(int device, int32_t** out) {
  if (device < 0 || device >= 64) return fail(PRECODE_EINVAL, "precode_solve_varlen_static: device");
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (!g_scratch_ptr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_varlen_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "precode_solve_varlen_static: cudaGetSymbolAddress");
    g_scratch_ptr[device] = static_cast<int32_t*>(p);
  }
  *out = g_scratch_ptr[device];
  return PRECODE_OK;
}

}  // namespace

}  // namespace precode

using namespace precode;

extern "C" precode_status_t precode_solve_varlen_static(
    const precode_desc_t* d, int64_t B, const precode_inst_t* tbl, const void* H, const float* t,
    const float* step, const float* lam, void* W, float* obj, float* resid, int32_t* flags,
    precode_stream_t stream) {
  if (!d) return fail(PRECODE_EINVAL, "precode_solve_varlen_static: NULL descriptor");
  if (d->mode != PRECODE_LAYER_PGD && d->mode != PRECODE_LAYER_PROJ)
    return fail(PRECODE_EINVAL, "precode_solve_varlen_static: unknown layer mode");
  if (d->T < 1 || d->T > PRECODE_MAX_T)
    return fail(PRECODE_EINVAL, "precode_solve_varlen_static: T out of range");
  if (d->flags & (PRECODE_PLAN_AUTOTUNE | PRECODE_PLAN_GRAPHS | PRECODE_PLAN_TENSOR_CORES))
    return fail(PRECODE_EINVAL,
                "precode_solve_varlen_static: autotuning, graphs and tensor-core buckets need a "
                "plan (precode_plan)");
  if ((d->flags & PRECODE_PLAN_STEP_NORMALISED) && d->mode != PRECODE_LAYER_PGD)
    return fail(PRECODE_EINVAL, "precode_solve_varlen_static: step normalisation is PGD-only");
  if (B < 0 || B > kMaxInst)
    return fail(PRECODE_EINVAL,
                "precode_solve_varlen_static: B must be in [0, PRECODE_STATIC_MAX_INSTANCES = 65536]");
  if (d->n_shapes < 1 || !d->shapes)
    return fail(PRECODE_EINVAL, "precode_solve_varlen_static: no shapes");
  if (B == 0) return PRECODE_OK;
  if (!tbl || !H || !t || !step || !W)
    return fail(PRECODE_EINVAL, "precode_solve_varlen_static: NULL buffer");
  if (d->mode == PRECODE_LAYER_PGD && !lam)
    return fail(PRECODE_EINVAL, "precode_solve_varlen_static: lam required for the paper layer");
  if (((uintptr_t)H & 15) || ((uintptr_t)W & 15) || ((uintptr_t)tbl & 7))
    return fail(PRECODE_EINVAL, "precode_solve_varlen_static: misaligned buffer");

  // buckets: each shape's default variant, plus the generic variant of each
  // bucket size (fixed-size tables, no allocation)
  StaticBuckets bt{};
  const Variant* bv[kMaxBk];
  bt.mode = d->mode;
  auto add = [&](int M, int K, const Variant* v) -> bool {
    for (int i = 0; i < bt.n; ++i)
      if (bv[i] == v && (!v->exact || (bt.M[i] == M && bt.K[i] == K))) return true;
    if (bt.n == kMaxBk) return false;
    bv[bt.n] = v;
    bt.M[bt.n] = M;
    bt.K[bt.n] = K;
    bt.KB[bt.n] = v->KB;
    bt.MB[bt.n] = v->MB;
    bt.exact[bt.n] = v->exact ? 1 : 0;
    ++bt.n;
    return true;
  };
  for (int i = 0; i < d->n_shapes; ++i) {
    const int M = d->shapes[i].M, K = d->shapes[i].K;
    if (!shape_ok(d->mode, M, K))
      return fail(PRECODE_EINVAL, "precode_solve_varlen_static: unsupported shape");
    const Variant* v = pick_variant(d->mode, M, K);
    if (!v) return fail(PRECODE_EINVAL, "precode_solve_varlen_static: no kernel bucket holds a shape");
    if (!add(M, K, v))
      return fail(PRECODE_EINVAL,
                  "precode_solve_varlen_static: more than PRECODE_STATIC_MAX_BUCKETS = 8 buckets");
  }
  const int nshape_buckets = bt.n;
  for (int i = 0; i < nshape_buckets; ++i) {
    if (!bv[i]->exact) continue;
    for (const auto& cand : variants())
      if (cand.mode == d->mode && !cand.exact && !cand.tc && cand.KB == bv[i]->KB &&
          cand.MB == bv[i]->MB) {
        if (!add(cand.MB, cand.KB, &cand))
          return fail(PRECODE_EINVAL,
                      "precode_solve_varlen_static: more than PRECODE_STATIC_MAX_BUCKETS = 8 buckets");
        break;
      }
  }

  DeviceGuard g(d->device);
  int32_t* scratch = nullptr;
  precode_status_t st = scratch_address(d->device, &scratch);
  if (st != PRECODE_OK) return st;
  int nsm = 0;
  cudaError_t e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, d->device);
  if (e != cudaSuccess) return cuda_fail(e, "precode_solve_varlen_static: device query");
  cudaStream_t s = (cudaStream_t)stream;
  // counters and the timeout counter start at zero on every call
  e = cudaMemsetAsync(scratch + kCountOff, 0, sizeof(int32_t) * (kWords - kCountOff), s);
  if (e != cudaSuccess) return cuda_fail(e, "precode_solve_varlen_static: clear counters");
  bucketize_static_kernel<<<2 * nsm, 256, 0, s>>>(reinterpret_cast<const InstDesc*>(tbl), B, bt,
                                                 scratch, flags);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "precode_solve_varlen_static: bucketing launch");
  for (int i = 0; i < bt.n; ++i) {
    const Variant* v = bv[i];
    e = cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v->smem);
    int occ = 0;
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, v->fn, v->threads, v->smem);
    if (e != cudaSuccess || occ <= 0)
      return fail(PRECODE_ECUDA, "precode_solve_varlen_static: kernel variant cannot run here");
    SolveArgs A{};
    A.H = static_cast<const float2*>(H);
    A.t = t;
    A.step = step;
    A.lam = lam ? lam : step;
    A.W = static_cast<float2*>(W);
    A.obj = obj;
    A.resid = resid;
    A.flags = flags;
    A.K = bt.K[i];
    A.M = bt.M[i];
    A.T = d->T;
    A.cond_thr = d->cond_threshold > 0 ? (float)d->cond_threshold : kDefaultCondThreshold;
    A.opts = (d->flags & PRECODE_PLAN_STEP_NORMALISED) ? OPT_STEP_NORMALISED : 0u;
    A.tbl = reinterpret_cast<const InstDesc*>(tbl);
    A.index = scratch + (int64_t)i * kMaxInst;
    A.count = scratch + kCountOff + i;
    A.err = reinterpret_cast<unsigned long long*>(scratch + kErrOff);
    void* args[] = {&A};
    e = cudaLaunchKernel(v->fn, dim3(occ * nsm), dim3(v->threads), args, (size_t)v->smem, s);
    if (e != cudaSuccess) return cuda_fail(e, "precode_solve_varlen_static: solve launch");
  }
  return PRECODE_OK;
}
