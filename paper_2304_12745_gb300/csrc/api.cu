// Host side of the C ABI: plans, argument validation, kernel-variant choice,
// launches, the host-buffer pipeline and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "api_internal.h"
#include "precode.h"
#include "registry.h"

namespace precode {

static thread_local std::string g_last_error;

precode_status_t fail(precode_status_t st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

precode_status_t cuda_fail(cudaError_t e, const char* what) {
  return fail(PRECODE_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Allocation-failure injection (PRECODE_INJECT_ENOMEM=N): true for the N-th call
// since the variable took its current value.
static bool inject_enomem() {
  static std::mutex mu;
  static std::string seen;
  static long long calls = 0;
  const char* v = std::getenv("PRECODE_INJECT_ENOMEM");
  std::lock_guard<std::mutex> lk(mu);
  if (!v || !*v) {
    seen.clear();
    return false;
  }
  if (seen != v) {
    seen = v;
    calls = 0;
  }
  const long long n = std::atoll(v);
  return n > 0 && ++calls == n;
}

cudaError_t dev_alloc(void** ptr, size_t bytes) {
  if (inject_enomem()) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(ptr, bytes);
}

cudaError_t pinned_alloc(void** ptr, size_t bytes) {
  if (inject_enomem()) {
    *ptr = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocHost(ptr, bytes);
}

const std::vector<Variant>& variants() {
  static std::vector<Variant> v = [] {
    std::vector<Variant> r;
    register_solve_pgd(r);
    register_solve_proj(r);
    register_solve_tch(r);  // before the TF32 build: the projected layer's default at 8 x 64
    register_solve_tc(r);
    register_solve_tcwh(r);  // before the TF32 builds: the projected layer's default there
    register_solve_tgt(r);  // before the row build: the default tcgen05 build
    register_solve_tg(r);
    register_solve_tcw_64(r);
    register_solve_tcw_128(r);
    register_solve_tcw_256(r);
    return r;
  }();
  return v;
}

// Blocks per SM a variant reaches on the current device (shared memory attribute set once).
int variant_occupancy(const Variant& v, int device) {
  static std::mutex mu;
  static std::vector<std::vector<int>> cache;  // [device][variant index]
  std::lock_guard<std::mutex> lk(mu);
  const auto& all = variants();
  const size_t idx = &v - all.data();
  if ((int)cache.size() <= device) cache.resize(device + 1);
  auto& c = cache[device];
  if (c.empty()) c.assign(all.size(), -1);
  if (c[idx] < 0) {
    if (cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem) !=
        cudaSuccess)
      return 0;
    cudaFuncSetAttribute(v.fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                         cudaSharedmemCarveoutMaxShared);
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, v.fn, v.threads, v.smem) != cudaSuccess)
      return 0;
    c[idx] = n;
  }
  return c[idx];
}

// Default choice: with tensor cores, the tcgen05 build where it holds (K, M) with
// fewer than 8 padded users, else the exact tensor-core build of (mode, K, M),
// else the smallest user-padded one with M antennas; then the first exact FP32
// variant, else the smallest generic bucket that holds (K, M).
const Variant* pick_variant(int mode, int M, int K, bool tensor_cores) {
  const Variant* best = nullptr;
  if (tensor_cores) {
    for (const auto& v : variants())
      if (v.tg && v.mode == mode && variant_fits(v, M, K) && v.KB < K + 8) return &v;
    for (const auto& v : variants())
      if (v.tc && v.exact && v.mode == mode && variant_fits(v, M, K)) return &v;
    for (const auto& v : variants())
      if (v.tc && !v.exact && v.mode == mode && variant_fits(v, M, K) && (!best || v.KB < best->KB))
        best = &v;
    if (best) return best;
  }
  for (const auto& v : variants())
    if (v.mode == mode && v.exact && !v.tc && variant_fits(v, M, K)) return &v;
  for (const auto& v : variants()) {
    if (v.mode != mode || v.exact || v.tc || !variant_fits(v, M, K)) continue;
    if (!best || v.KB * v.MB < best->KB * best->MB) best = &v;
  }
  return best;
}

// Autotuning candidates: every variant that fits, except user-padded tensor-core
// builds with 8 or more padded users (never faster than the tighter build).
std::vector<const Variant*> eligible_variants(int mode, int M, int K) {
  std::vector<const Variant*> r;
  for (const auto& v : variants())
    if (v.mode == mode && variant_fits(v, M, K) && (!v.tc || v.exact || v.KB < K + 8))
      r.push_back(&v);
  return r;
}

DeviceGuard::DeviceGuard(int dev) {
  cudaGetDevice(&prev_);
  if (prev_ != dev) cudaSetDevice(dev);
}
DeviceGuard::~DeviceGuard() {
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != prev_) cudaSetDevice(prev_);
}

precode_status_t launch_variant(const Variant& v, int device, int num_sms, const SolveArgs& A,
                                int64_t n_hint, cudaStream_t stream) {
  const int occ = variant_occupancy(v, device);
  if (occ <= 0) return fail(PRECODE_ECUDA, "kernel variant cannot be resident on this device");
  int64_t grid = (int64_t)occ * num_sms;
  if (n_hint >= 0) grid = std::min<int64_t>(grid, (n_hint + v.groups - 1) / v.groups);
  if (grid < 1) grid = 1;
  SolveArgs a = A;
  void* args[] = {&a};
  cudaError_t e = cudaLaunchKernel(v.fn, dim3((unsigned)grid), dim3(v.threads), args,
                                   (size_t)v.smem, stream);
  if (e != cudaSuccess) return cuda_fail(e, "solve kernel launch");
  return PRECODE_OK;
}

bool shape_ok(int mode, int M, int K) {
  if (K < 1 || K > PRECODE_MAX_K || M < 2 || M > PRECODE_MAX_M || (M & 1)) return false;
  if (mode == PRECODE_LAYER_PROJ && K > M) return false;
  return true;
}

}  // namespace precode

using namespace precode;

namespace precode {
void plan_build_buckets(precode_plan_t p) {
  p->buckets.clear();
  auto add = [&](int M, int K, const Variant* v) {
    for (const auto& b : p->buckets)
      if (b.v == v && (!v->exact || (b.M == M && b.K == K))) return;
    p->buckets.push_back(Bucket{M, K, v});
  };
  for (size_t i = 0; i < p->shapes.size(); ++i) add(p->shapes[i].M, p->shapes[i].K, p->chosen[i]);
  // Every bucket also gets the generic FP32 build of its (KB, MB), so any shape
  // that fits the bucket has a kernel (a tensor-core build needs M == MB), and an
  // exact tensor-core bucket its user-padded tensor-core build.
  const size_t n = p->buckets.size();
  for (size_t i = 0; i < n; ++i) {
    const Variant* v = p->buckets[i].v;
    for (const auto& cand : variants()) {
      if (cand.mode != p->mode || cand.exact || cand.KB != v->KB || cand.MB != v->MB) continue;
      if (!cand.tc || (v->tc && v->exact)) add(cand.MB, cand.KB, &cand);
    }
  }
}
}  // namespace precode

static void plan_free(precode_plan_t p) {
  if (!p) return;
  DeviceGuard g(p->device);
  if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  cudaFree(p->d_index);
  cudaFree(p->d_count);
  cudaFree(p->d_cp);
  cudaFree(p->d_part);
  if (p->d_err) cudaFree(p->d_err);
  for (int i = 0; i < precode_plan_s::kPipe; ++i) {
    if (p->hstream[i]) cudaStreamDestroy(p->hstream[i]);
    cudaFree(p->dH[i]);
    cudaFree(p->dW[i]);

  }
  cudaFree(p->dparams);
  cudaFree(p->dt_all);
  cudaFree(p->dobj_all);
  cudaFree(p->dres_all);
  cudaFree(p->dfl_all);
  for (auto& ev : p->hev)
    if (ev) cudaEventDestroy(ev);
  delete p;
}

namespace precode {
precode_status_t autotune_plan(precode_plan_t p, const char* cache_path);
}  // namespace precode

precode_status_t precode::plan_export_factors(precode_plan_t p, int32_t M, int32_t K, int64_t n,
                                              const void* H, float2* fac, void* W, const float* t,
                                              cudaStream_t stream, int* stride) {
  *stride = 0;
  if (!p || n < 1 || !H || !fac || !W || !t || p->mode != PRECODE_LAYER_PROJ || !shape_ok(p->mode, M, K))
    return PRECODE_OK;
  const Variant* v = p->variant_for(M, K);
  if (!v || !v->fac) return PRECODE_OK;
  std::lock_guard<std::mutex> lk(p->mu);
  DeviceGuard g(p->device);
  SolveArgs A{};
  A.H = static_cast<const float2*>(H);
  A.t = t;
  A.t_stride = 0;
  A.step = t;  // not read: no layers
  A.lam = t;
  A.W = static_cast<float2*>(W);
  A.B = n;
  A.K = K;
  A.M = M;
  A.T = 0;
  A.cond_thr = p->cond_thr;
  A.opts = p->kernel_opts() | OPT_FAC_EXPORT;
  A.wait_ns = p->wait_ns;
  A.err = p->d_err;
  A.fac = fac;
  const precode_status_t st = launch_variant(*v, p->device, p->num_sms, A, n, stream);
  if (st == PRECODE_OK) *stride = fac_stride(v->KB);
  return st;
}

extern "C" {

const char* precode_status_str(precode_status_t s) {
  switch (s) {
    case PRECODE_OK: return "ok";
    case PRECODE_EINVAL: return "invalid argument";
    case PRECODE_ENOMEM: return "out of memory";
    case PRECODE_ECUDA: return "CUDA error";
    case PRECODE_ETIMEDOUT: return "timed out";
    case PRECODE_EBUSY: return "busy";
    case PRECODE_PENDING: return "pending";
    case PRECODE_ENOTFOUND: return "not found";
  }
  return "unknown status";
}

const char* precode_last_error(void) { return g_last_error.c_str(); }

precode_status_t precode_plan(const precode_desc_t* d, precode_plan_t* out) {
  try {
    if (!d || !out) return fail(PRECODE_EINVAL, "precode_plan: NULL argument");
    *out = nullptr;
    if (d->mode != PRECODE_LAYER_PGD && d->mode != PRECODE_LAYER_PROJ)
      return fail(PRECODE_EINVAL, "precode_plan: unknown layer mode");
    if (d->T < 1 || d->T > PRECODE_MAX_T) return fail(PRECODE_EINVAL, "precode_plan: T out of range");
    if (d->n_shapes < 1 || !d->shapes) return fail(PRECODE_EINVAL, "precode_plan: no shapes");
    if (d->max_instances < 1) return fail(PRECODE_EINVAL, "precode_plan: max_instances < 1");
    if ((d->flags & PRECODE_PLAN_STEP_NORMALISED) && d->mode != PRECODE_LAYER_PGD)
      return fail(PRECODE_EINVAL, "precode_plan: step normalisation applies to the paper layer");
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "precode_plan: no CUDA device");
    if (d->device < 0 || d->device >= ndev) return fail(PRECODE_EINVAL, "precode_plan: bad device");
    std::unique_ptr<precode_plan_s, void (*)(precode_plan_t)> p(new precode_plan_s, plan_free);
    p->mode = d->mode;
    p->T = d->T;
    p->device = d->device;
    p->max_instances = d->max_instances;
    p->cond_thr = d->cond_threshold > 0 ? (float)d->cond_threshold : kDefaultCondThreshold;
    p->flags = d->flags;
    DeviceGuard g(p->device);
    e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return cuda_fail(e, "precode_plan: device query");
    for (int i = 0; i < d->n_shapes; ++i) {
      const auto s = d->shapes[i];
      if (!shape_ok(d->mode, s.M, s.K))
        return fail(PRECODE_EINVAL, "precode_plan: shape (M=" + std::to_string(s.M) + ", K=" +
                                        std::to_string(s.K) + ") unsupported");
      const Variant* v = pick_variant(d->mode, s.M, s.K, (d->flags & PRECODE_PLAN_TENSOR_CORES) != 0);
      if (!v) return fail(PRECODE_EINVAL, "precode_plan: no kernel bucket holds the shape");
      if (variant_occupancy(*v, p->device) <= 0)
        return fail(PRECODE_ECUDA, "precode_plan: kernel variant cannot run on this device");
      p->shapes.push_back(s);
      p->chosen.push_back(v);
    }
    e = dev_alloc(&p->d_err, sizeof(unsigned long long));
    if (e != cudaSuccess) return fail(PRECODE_ENOMEM, "precode_plan: device allocation");
    e = cudaMemset(p->d_err, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(e, "precode_plan: memset");
    if (d->flags & PRECODE_PLAN_AUTOTUNE) {
      precode_status_t st = autotune_plan(p.get(), d->tune_cache);
      if (st != PRECODE_OK) return st;
    }
    plan_build_buckets(p.get());
    for (const auto& b : p->buckets)
      if (variant_occupancy(*b.v, p->device) <= 0)
        return fail(PRECODE_ECUDA, "precode_plan: bucket variant cannot run on this device");
    *out = p.release();
    return PRECODE_OK;
  } catch (const std::exception& ex) {
    return fail(PRECODE_ENOMEM, std::string("precode_plan: ") + ex.what());
  }
}

precode_status_t precode_plan_destroy(precode_plan_t plan) {
  if (!plan) return fail(PRECODE_EINVAL, "precode_plan_destroy: NULL plan");
  plan_free(plan);
  return PRECODE_OK;
}

precode_status_t precode_solve(precode_plan_t p, int32_t M, int32_t K, int64_t B, const void* H,
                               const float* t, int64_t t_stride, const float* step,
                               const float* lam, void* W, float* obj, float* resid,
                               int32_t* flags, precode_stream_t stream) {
  if (!p) return fail(PRECODE_EINVAL, "precode_solve: NULL plan");
  if (B < 0 || B > p->max_instances)
    return fail(PRECODE_EINVAL, "precode_solve: B outside [0, max_instances]");
  if (!shape_ok(p->mode, M, K)) return fail(PRECODE_EINVAL, "precode_solve: unsupported shape");
  if (B == 0) return PRECODE_OK;
  if (!H || !t || !step || !W) return fail(PRECODE_EINVAL, "precode_solve: NULL buffer");
  if (p->mode == PRECODE_LAYER_PGD && !lam)
    return fail(PRECODE_EINVAL, "precode_solve: lam required for the paper layer");
  if (((uintptr_t)H & 15) || ((uintptr_t)W & 15))
    return fail(PRECODE_EINVAL, "precode_solve: H and W must be 16-byte aligned");
  if (t_stride != 0 && t_stride < K) return fail(PRECODE_EINVAL, "precode_solve: t_stride < K");
  const Variant* v = p->variant_for(M, K);
  if (!v) return fail(PRECODE_EINVAL, "precode_solve: shape not covered by the plan");
  DeviceGuard g(p->device);
  SolveArgs A{};
  A.H = static_cast<const float2*>(H);
  A.t = t;
  A.t_stride = t_stride;
  A.step = step;
  A.lam = lam ? lam : step;
  A.W = static_cast<float2*>(W);
  A.obj = obj;
  A.resid = resid;
  A.flags = flags;
  A.B = B;
  A.K = K;
  A.M = M;
  A.T = p->T;
  A.cond_thr = p->cond_thr;
  A.opts = p->kernel_opts();
  A.wait_ns = p->wait_ns;
  A.err = p->d_err;
  return launch_variant(*v, p->device, p->num_sms, A, B, (cudaStream_t)stream);
}

precode_status_t precode_solve_host(precode_plan_t p, int32_t M, int32_t K, int64_t B,
                                    const void* H, const float* t, int64_t t_stride,
                                    const float* step, const float* lam, void* W, float* obj,
                                    float* resid, int32_t* flags) {
  if (!p) return fail(PRECODE_EINVAL, "precode_solve_host: NULL plan");
  if (B < 0 || B > p->max_instances)
    return fail(PRECODE_EINVAL, "precode_solve_host: B outside [0, max_instances]");
  if (!shape_ok(p->mode, M, K)) return fail(PRECODE_EINVAL, "precode_solve_host: bad shape");
  if (B == 0) return PRECODE_OK;
  if (!H || !t || !step || !W) return fail(PRECODE_EINVAL, "precode_solve_host: NULL buffer");
  if (p->mode == PRECODE_LAYER_PGD && !lam)
    return fail(PRECODE_EINVAL, "precode_solve_host: lam required for the paper layer");
  if (t_stride != 0 && t_stride < K)
    return fail(PRECODE_EINVAL, "precode_solve_host: t_stride < K");
  if (!p->variant_for(M, K)) return fail(PRECODE_EINVAL, "precode_solve_host: shape not in plan");
  std::lock_guard<std::mutex> lk(p->mu);
  DeviceGuard g(p->device);
  cudaError_t e;
  if (!p->dparams) {
    e = dev_alloc(&p->dparams, sizeof(float) * 2 * p->T);
    if (e != cudaSuccess) return fail(PRECODE_ENOMEM, "precode_solve_host: params buffer");
  }
  // Zero-copy: when every buffer is page-locked host memory mapped into the
  // device's address space and the shape runs on the projected layer's split-FP16
  // K = 8 build, its host-buffer twin reads H and writes W over the host link from
  // inside the kernel (no staging copies; both directions overlap the solve).  The
  // twins are projected-layer builds: the paper layer takes the staged pipeline.
  {
    const Variant* v = p->variant_for(M, K);
    const void* hfn = (p->mode == PRECODE_LAYER_PROJ && v->mode == PRECODE_LAYER_PROJ && v->f16 &&
                       v->exact && v->KB == 8 && v->MB == 64)
                          ? tch_host_kernel(v->NW, v->minb) : nullptr;
    auto mapped = [](const void* ptr, void** dptr) -> bool {
      cudaPointerAttributes a{};
      if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
      }
      if (a.type != cudaMemoryTypeHost || !a.devicePointer) return false;
      *dptr = a.devicePointer;
      return true;
    };
    void *dH = nullptr, *dW = nullptr, *dt = nullptr, *dob = nullptr, *drs = nullptr, *dfl = nullptr;
    const bool zc = hfn && mapped(H, &dH) && mapped(W, &dW) && mapped(t, &dt) &&
                    (!obj || mapped(obj, &dob)) && (!resid || mapped(resid, &drs)) &&
                    (!flags || mapped(flags, &dfl)) && (uintptr_t)dH % 16 == 0 &&
                    (uintptr_t)dW % 16 == 0;
    if (zc) {
      if (!p->hstream[0] &&
          cudaStreamCreateWithFlags(&p->hstream[0], cudaStreamNonBlocking) != cudaSuccess)
        return fail(PRECODE_ECUDA, "precode_solve_host: stream");
      e = cudaMemcpy(p->dparams, step, sizeof(float) * p->T, cudaMemcpyHostToDevice);
      if (e == cudaSuccess && lam)
        e = cudaMemcpy(p->dparams + p->T, lam, sizeof(float) * p->T, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) return cuda_fail(e, "precode_solve_host: params copy");
      int occ = 0;
      e = cudaFuncSetAttribute(hfn, cudaFuncAttributeMaxDynamicSharedMemorySize, v->smem);
      if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, hfn, v->threads, v->smem);
      if (e != cudaSuccess || occ <= 0) return cuda_fail(e, "precode_solve_host: host-buffer kernel");
      SolveArgs A{};
      A.H = static_cast<const float2*>(dH);
      A.t = static_cast<const float*>(dt);
      A.t_stride = t_stride;
      A.step = p->dparams;
      A.lam = lam ? p->dparams + p->T : p->dparams;
      A.W = static_cast<float2*>(dW);
      A.obj = static_cast<float*>(dob);
      A.resid = static_cast<float*>(drs);
      A.flags = static_cast<int32_t*>(dfl);
      A.B = B;
      A.K = K;
      A.M = M;
      A.T = p->T;
      A.cond_thr = p->cond_thr;
      A.opts = p->kernel_opts();
      A.wait_ns = p->wait_ns;
      A.err = p->d_err;
      const int64_t grid = std::max<int64_t>(
          1, std::min<int64_t>((int64_t)occ * p->num_sms, (B + v->groups - 1) / v->groups));
      void* args[] = {&A};
      e = cudaLaunchKernel(hfn, dim3((unsigned)grid), dim3(v->threads), args, (size_t)v->smem,
                           p->hstream[0]);
      if (e == cudaSuccess) e = cudaStreamSynchronize(p->hstream[0]);
      if (e != cudaSuccess) return cuda_fail(e, "precode_solve_host: host-buffer solve");
      return PRECODE_OK;
    }
  }
  const size_t n = (size_t)K * M;
  // Chunks rotate over kPipe streams, each stream running copy in -> solve ->
  // copy out for its chunks, so the copy in of chunk c + 1, the solve of chunk c
  // and the copy out of chunk c - 1 overlap (the host link is the bound: both
  // copy directions together are slower than the solve).  At most 16 chunks, at
  // least 4,096 instances each.  The targets go in, and the per-instance outputs
  // come back, as one copy per call each (many small copies cost the copy
  // engines more than their bytes).
  int64_t chunk = std::max<int64_t>(std::min<int64_t>(B, 4096), (B + 15) / 16);
  if ((size_t)chunk * n > p->chunk_elems || chunk > p->chunk) {
    for (int i = 0; i < precode_plan_s::kPipe; ++i) {
      cudaFree(p->dH[i]);
      cudaFree(p->dW[i]);
      p->dH[i] = p->dW[i] = nullptr;
    }
    p->chunk = std::max<int64_t>(chunk, p->chunk);
    p->chunk_elems = std::max<size_t>((size_t)chunk * n, p->chunk_elems);
    for (int i = 0; i < precode_plan_s::kPipe; ++i) {
      if (dev_alloc(&p->dH[i], p->chunk_elems * 8) != cudaSuccess ||
          dev_alloc(&p->dW[i], p->chunk_elems * 8) != cudaSuccess)
        return fail(PRECODE_ENOMEM, "precode_solve_host: staging buffers");
      if (!p->hstream[i] &&
          cudaStreamCreateWithFlags(&p->hstream[i], cudaStreamNonBlocking) != cudaSuccess)
        return fail(PRECODE_ECUDA, "precode_solve_host: stream");
    }
  }
  for (auto& ev : p->hev)
    if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
      return fail(PRECODE_ECUDA, "precode_solve_host: event");
  const int64_t t_elems = t_stride ? B * t_stride : K;
  if (t_elems > p->t_cap) {
    cudaFree(p->dt_all);
    p->dt_all = nullptr;
    if (dev_alloc(&p->dt_all, (size_t)t_elems * 4) != cudaSuccess)
      return fail(PRECODE_ENOMEM, "precode_solve_host: target buffer");
    p->t_cap = t_elems;
  }
  if (B > p->out_cap) {
    cudaFree(p->dobj_all);
    cudaFree(p->dres_all);
    cudaFree(p->dfl_all);
    p->dobj_all = p->dres_all = nullptr;
    p->dfl_all = nullptr;
    if (dev_alloc(&p->dobj_all, (size_t)B * 4) != cudaSuccess ||
        dev_alloc(&p->dres_all, (size_t)B * 4) != cudaSuccess ||
        dev_alloc(&p->dfl_all, (size_t)B * 4) != cudaSuccess)
      return fail(PRECODE_ENOMEM, "precode_solve_host: output buffers");
    p->out_cap = B;
  }
  e = cudaMemcpy(p->dparams, step, sizeof(float) * p->T, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && lam)
    e = cudaMemcpy(p->dparams + p->T, lam, sizeof(float) * p->T, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "precode_solve_host: params copy");
  // targets once, on stream 0; the other streams wait for them
  cudaStream_t S0 = p->hstream[0];
  e = cudaMemcpyAsync(p->dt_all, t, (size_t)t_elems * 4, cudaMemcpyHostToDevice, S0);
  if (e == cudaSuccess) e = cudaEventRecord(p->hev[precode_plan_s::kPipe], S0);
  for (int i = 1; i < precode_plan_s::kPipe && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(p->hstream[i], p->hev[precode_plan_s::kPipe], 0);
  if (e != cudaSuccess) return cuda_fail(e, "precode_solve_host: targets copy");
  const char* Hc = static_cast<const char*>(H);
  char* Wc = static_cast<char*>(W);
  precode_status_t st = PRECODE_OK;
  for (int64_t c0 = 0, ci = 0; c0 < B; c0 += chunk, ++ci) {
    const int s = (int)(ci % precode_plan_s::kPipe);
    cudaStream_t S = p->hstream[s];
    const int64_t nb = std::min<int64_t>(chunk, B - c0);
    e = cudaMemcpyAsync(p->dH[s], Hc + (size_t)c0 * n * 8, (size_t)nb * n * 8,
                        cudaMemcpyHostToDevice, S);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "precode_solve_host: copy in");
      break;
    }
    st = precode_solve(p, M, K, nb, p->dH[s], t_stride ? p->dt_all + c0 * t_stride : p->dt_all,
                       t_stride, p->dparams, lam ? p->dparams + p->T : nullptr, p->dW[s],
                       obj ? p->dobj_all + c0 : nullptr, resid ? p->dres_all + c0 : nullptr,
                       flags ? p->dfl_all + c0 : nullptr, S);
    if (st != PRECODE_OK) break;
    e = cudaMemcpyAsync(Wc + (size_t)c0 * n * 8, p->dW[s], (size_t)nb * n * 8,
                        cudaMemcpyDeviceToHost, S);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "precode_solve_host: copy out");
      break;
    }
  }
  // per-instance outputs: stream 0 waits for every stream, then one copy each
  if (st == PRECODE_OK) {
    for (int i = 1; i < precode_plan_s::kPipe && e == cudaSuccess; ++i) {
      e = cudaEventRecord(p->hev[i], p->hstream[i]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(S0, p->hev[i], 0);
    }
    if (e == cudaSuccess && obj)
      e = cudaMemcpyAsync(obj, p->dobj_all, (size_t)B * 4, cudaMemcpyDeviceToHost, S0);
    if (e == cudaSuccess && resid)
      e = cudaMemcpyAsync(resid, p->dres_all, (size_t)B * 4, cudaMemcpyDeviceToHost, S0);
    if (e == cudaSuccess && flags)
      e = cudaMemcpyAsync(flags, p->dfl_all, (size_t)B * 4, cudaMemcpyDeviceToHost, S0);
    if (e != cudaSuccess) st = cuda_fail(e, "precode_solve_host: outputs copy");
  }
  for (int i = 0; i < precode_plan_s::kPipe; ++i) {
    e = cudaStreamSynchronize(p->hstream[i]);
    if (e != cudaSuccess && st == PRECODE_OK) st = cuda_fail(e, "precode_solve_host: sync");
  }
  return st;
}

precode_status_t precode_plan_describe(precode_plan_t p, int32_t M, int32_t K, char* buf,
                                       size_t len) {
  if (!p || !buf || len == 0) return fail(PRECODE_EINVAL, "precode_plan_describe: bad argument");
  const Variant* v = p->variant_for(M, K);
  if (!v) return fail(PRECODE_EINVAL, "precode_plan_describe: shape not covered by the plan");
  if (v->tgt)
    std::snprintf(buf, len, "solve_tgt_kernel<%d>", v->minb);
  else if (v->tg)
    std::snprintf(buf, len, "solve_tg_kernel<%d>", v->minb);
  else if (v->f16 && v->exact && v->KB == 8 && v->MB == 64 && v->mode == PRECODE_LAYER_PGD)
    std::snprintf(buf, len, "solve_tch_kernel<%d, %d, 0, 0>", v->NW, v->minb);
  else if (v->f16 && v->exact && v->KB == 8 && v->MB == 64)
    std::snprintf(buf, len, "solve_tch_kernel<%d, %d>", v->NW, v->minb);
  else if (v->f16)
    std::snprintf(buf, len, "solve_tcwh_kernel<%d, %d, %d>", v->NW, v->MB, v->minb);
  else if (v->tc && v->exact && v->KB == 8 && v->MB == 64)
    std::snprintf(buf, len, "solve_tc_kernel<%d, %d, %d, %d>", v->mode, v->NW, v->minb,
                  v->db ? 1 : 0);
  else if (v->tc)
    std::snprintf(buf, len, "solve_tcw_kernel<%d, %d, %d, %d>", v->mode, v->NW, v->MB, v->minb);
  else
    std::snprintf(buf, len, "solve_kernel<%d, %d, %d, %d, %d, %d, %d, %d, %d, %d, %d>", v->mode,
                  v->KB, v->MB, v->GK, v->GM, v->JC, v->exact ? 1 : 0, v->NW, v->minb,
                  v->split ? 1 : 0, v->db ? 1 : 0);
  return PRECODE_OK;
}

precode_status_t precode_plan_set_debug(precode_plan_t p, uint64_t wait_limit_ns,
                                        int32_t inject_copy_stall) {
  if (!p) return fail(PRECODE_EINVAL, "precode_plan_set_debug: NULL plan");
  std::lock_guard<std::mutex> lk(p->mu);
  p->wait_ns = wait_limit_ns;
  p->stall_copy = inject_copy_stall != 0;
  return PRECODE_OK;
}

precode_status_t precode_plan_errors(precode_plan_t p, uint64_t* count) {
  if (!p || !count) return fail(PRECODE_EINVAL, "precode_plan_errors: NULL argument");
  DeviceGuard g(p->device);
  unsigned long long v = 0;
  cudaError_t e = cudaMemcpy(&v, p->d_err, sizeof(v), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "precode_plan_errors");
  *count = v;
  return PRECODE_OK;
}

}  // extern "C"
