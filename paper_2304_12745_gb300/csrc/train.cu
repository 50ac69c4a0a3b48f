// precode_train_step: forward + adjoint through the T layers of a uniform batch,
// then a deterministic FP64 batch mean of the per-instance loss and gradients.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <map>
#include <mutex>
#include <utility>

#include "api_internal.h"
#include "train.cuh"

namespace precode {

const std::vector<TrainVariant>& train_variants() {
  static std::vector<TrainVariant> v = [] {
    std::vector<TrainVariant> r;
    register_train_pgd(r);
    register_train_proj(r);
    register_train_tch(r);  // before the TF32 build: the projected layer's default at 8 x 64
    register_train_tc(r);
    return r;
  }();
  return v;
}

namespace {

// Batch means of the per-instance partials part[b][j] (j = 0: loss, 1..T: d step,
// T+1..2T: d lam), in FP64 and in an order fixed by B and P alone, so a step gives the
// same bits on every run.  Stage 1: block g sums rows [g R, (g+1) R) of every column;
// for P <= 256 its threads read whole rows (coalesced), thread i taking column i % P of
// every (256 / P)-th row, and the row phases are then added in order.  Stage 2: one
// block per column adds the G block sums (strided, then a fixed tree) and scales.
constexpr int kSumThreads = 256;

struct BatchSumShape {
  int64_t rows;  // R: rows per stage-1 block
  int blocks;    // G = ceil(B / R) <= bound
  int bound;     // non-decreasing in B: sizes the block-sum scratch for every B <= B_max
};

BatchSumShape batch_sum_shape(int64_t B, int P) {
  int64_t g = (B + kSumThreads - 1) / kSumThreads;
  g = std::min<int64_t>(g, 1024);
  g = std::min<int64_t>(g, std::max<int64_t>(1, (int64_t(1) << 22) / P));
  const int64_t rows = (B + g - 1) / g;
  return {rows, (int)((B + rows - 1) / rows), (int)g};
}

__global__ void __launch_bounds__(kSumThreads)
batch_sum_rows_kernel(const float* __restrict__ part, int64_t B, int P, int64_t rows,
                      double* __restrict__ bsum) {
  __shared__ double buf[kSumThreads];
  const int64_t r0 = (int64_t)blockIdx.x * rows;
  const int64_t r1 = r0 + rows < B ? r0 + rows : B;
  double* out = bsum + (int64_t)blockIdx.x * P;
  const int i = threadIdx.x;
  if (P <= kSumThreads) {
    const int rpp = kSumThreads / P;
    double s = 0.0;
    if (i < rpp * P) {
      const int j = i % P;
#pragma unroll 4
      for (int64_t r = r0 + i / P; r < r1; r += rpp) s += (double)part[r * P + j];
    }
    buf[i] = s;
    __syncthreads();
    if (i < P) {
      double t = 0.0;
      for (int q = 0; q < rpp; ++q) t += buf[q * P + i];
      out[i] = t;
    }
  } else {
    for (int j = i; j < P; j += kSumThreads) {
      double s = 0.0;
      for (int64_t r = r0; r < r1; ++r) s += (double)part[r * P + j];
      out[j] = s;
    }
  }
}

__global__ void __launch_bounds__(kSumThreads)
batch_sum_finish_kernel(const double* __restrict__ bsum, int G, int P, int T, double scale,
                        float* __restrict__ loss, float* __restrict__ dstep,
                        float* __restrict__ dlam) {
  __shared__ double buf[kSumThreads];
  const int j = blockIdx.x;
  double s = 0.0;
  for (int g = threadIdx.x; g < G; g += kSumThreads) s += bsum[(int64_t)g * P + j];
  buf[threadIdx.x] = s;
  __syncthreads();
  for (int span = kSumThreads / 2; span > 0; span >>= 1) {
    if ((int)threadIdx.x < span) buf[threadIdx.x] += buf[threadIdx.x + span];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const float v = (float)(buf[0] * scale);
    if (j == 0)
      *loss = v;
    else if (j <= T)
      dstep[j - 1] = v;
    else
      dlam[j - 1 - T] = v;
  }
}


const TrainVariant* pick_train(int mode, int M, int K, bool tensor_cores) {
  const TrainVariant* best = nullptr;
  // PRECODE_TRAIN_TF32 set: the split-TF32 tensor-core build even where a split-FP16
  // one exists (comparison and testing)
  const bool tf32_only = std::getenv("PRECODE_TRAIN_TF32") != nullptr;
  if (tensor_cores)
    for (const auto& v : train_variants())
      if (v.tc && !(tf32_only && v.f16) && v.mode == mode && v.exact && v.KB == K && v.MB == M)
        return &v;
  for (const auto& v : train_variants())
    if (!v.tc && v.mode == mode && v.exact && v.KB == K && v.MB == M) return &v;
  for (const auto& v : train_variants()) {
    if (v.tc || v.mode != mode || v.exact || v.KB < K || v.MB < M) continue;
    if (!best || v.KB * v.MB < best->KB * best->MB) best = &v;
  }
  return best;
}

// Resident blocks per SM, set up and queried once per kernel and device: later
// steps make no attribute or occupancy calls, so a step can be captured into a
// CUDA graph after its first eager run.
int train_occupancy(const TrainVariant& v, int device) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, int> cache;
  std::lock_guard<std::mutex> lk(mu);
  const auto key = std::make_pair(v.fn, device);
  const auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (cudaFuncSetAttribute(v.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, v.smem) !=
      cudaSuccess)
    return 0;
  cudaFuncSetAttribute(v.fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                       cudaSharedmemCarveoutMaxShared);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, v.fn, v.threads, v.smem) != cudaSuccess)
    return 0;
  cache[key] = n;
  return n;
}

}  // namespace

}  // namespace precode

using namespace precode;

// Forward + adjoint launch and batch reductions shared by the unsupervised
// (wgt == nullptr, weight a) and the supervised (labels wgt) train steps.
static precode_status_t train_step_impl(precode_plan_t p, int32_t M, int32_t K, int64_t B,
                                        const void* H, const float* t, int64_t t_stride,
                                        const float* step, const float* lam, float a,
                                        const void* wgt, float* loss, float* dstep, float* dlam,
                                        int32_t* flags, precode_stream_t stream) {
  if (!p) return fail(PRECODE_EINVAL, "precode_train_step: NULL plan");
  if (B < 1 || B > p->max_instances)
    return fail(PRECODE_EINVAL, "precode_train_step: B outside [1, max_instances]");
  if (!shape_ok(p->mode, M, K)) return fail(PRECODE_EINVAL, "precode_train_step: bad shape");
  if (!H || !t || !step || !loss || !dstep)
    return fail(PRECODE_EINVAL, "precode_train_step: NULL buffer");
  if (p->mode == PRECODE_LAYER_PGD && (!lam || !dlam))
    return fail(PRECODE_EINVAL, "precode_train_step: lam and dlam required for the paper layer");
  if ((uintptr_t)H & 15) return fail(PRECODE_EINVAL, "precode_train_step: H must be 16-byte aligned");
  if ((uintptr_t)wgt & 15)
    return fail(PRECODE_EINVAL, "precode_train_step_supervised: W_gt must be 16-byte aligned");
  if (t_stride != 0 && t_stride < K) return fail(PRECODE_EINVAL, "precode_train_step: t_stride < K");
  const TrainVariant* v = pick_train(p->mode, M, K, (p->flags & PRECODE_PLAN_TENSOR_CORES) != 0);
  if (!v) return fail(PRECODE_EINVAL, "precode_train_step: no train kernel holds the shape");
  std::lock_guard<std::mutex> lk(p->mu);
  DeviceGuard g(p->device);
  const int T = p->T;
  // checkpoint interval: ceil(sqrt(T)), or the shortest interval whose checkpoints
  // all fit in the kernel's tensor memory when that is shorter (fewer layers
  // recomputed in the reverse pass)
  int cpe = (int)std::ceil(std::sqrt((double)T));
  if (v->cp_onchip > 0) {
    const int c_chip = (T + v->cp_onchip - 1) / v->cp_onchip;
    if (c_chip < cpe) cpe = c_chip;
  }
  const int ncp = (T + cpe - 1) / cpe;
  // checkpoints in tensor memory where the kernel holds them, else a global workspace
  const bool cp_onchip = ncp <= v->cp_onchip;
  const size_t cp_need =
      cp_onchip ? 0 : (size_t)p->max_instances * ncp * v->KB * v->MB * sizeof(float2);
  // per-instance partials, then (8-byte aligned) the stage-1 block sums of the batch means
  const int PW = 1 + 2 * T;
  const size_t part_floats = ((size_t)p->max_instances * PW + 1) & ~(size_t)1;
  const size_t part_need = part_floats * sizeof(float) +
                           (size_t)batch_sum_shape(p->max_instances, PW).bound * PW * sizeof(double);
  if (cp_need > p->cp_bytes) {
    cudaFree(p->d_cp);
    p->d_cp = nullptr;
    p->cp_bytes = 0;
    if (dev_alloc(&p->d_cp, cp_need) != cudaSuccess)
      return fail(PRECODE_ENOMEM, "precode_train_step: checkpoint workspace");
    p->cp_bytes = cp_need;
  }
  if (part_need > p->part_bytes) {
    cudaFree(p->d_part);
    p->d_part = nullptr;
    p->part_bytes = 0;
    if (dev_alloc(&p->d_part, part_need) != cudaSuccess)
      return fail(PRECODE_ENOMEM, "precode_train_step: gradient workspace");
    p->part_bytes = part_need;
  }
  const int occ = train_occupancy(*v, p->device);
  if (occ <= 0) return fail(PRECODE_ECUDA, "precode_train_step: kernel cannot run on this device");
  TrainArgs A{};
  A.s.H = static_cast<const float2*>(H);
  A.s.t = t;
  A.s.t_stride = t_stride;
  A.s.step = step;
  A.s.lam = lam ? lam : step;
  A.s.flags = flags;
  A.s.B = B;
  A.s.K = K;
  A.s.M = M;
  A.s.T = T;
  A.s.cond_thr = p->cond_thr;
  A.s.opts = p->kernel_opts();
  A.s.wait_ns = p->wait_ns;
  A.s.err = p->d_err;
  A.a = a;
  A.wgt = static_cast<const float2*>(wgt);
  A.cp = cp_onchip ? nullptr : p->d_cp;
  A.cp_every = cpe;
  A.ncp = ncp;
  A.part = p->d_part;
  cudaStream_t s = (cudaStream_t)stream;
  int64_t grid = std::min<int64_t>((int64_t)occ * p->num_sms, (B + v->groups - 1) / v->groups);
  void* args[] = {&A};
  cudaError_t e = cudaLaunchKernel(v->fn, dim3((unsigned)grid), dim3(v->threads), args,
                                   (size_t)v->smem, s);
  if (e != cudaSuccess) return cuda_fail(e, "precode_train_step: train kernel launch");
  // loss (column 0), d step (columns 1..T) and, where asked for, d lam (T+1..2T)
  const BatchSumShape bs = batch_sum_shape(B, PW);
  double* bsum = reinterpret_cast<double*>(p->d_part + part_floats);
  batch_sum_rows_kernel<<<bs.blocks, kSumThreads, 0, s>>>(p->d_part, B, PW, bs.rows, bsum);
  batch_sum_finish_kernel<<<dlam ? PW : 1 + T, kSumThreads, 0, s>>>(
      bsum, bs.blocks, PW, T, 1.0 / (double)B, loss, dstep, dlam);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "precode_train_step: batch reduction launch");
  return PRECODE_OK;
}

extern "C" precode_status_t precode_train_step(precode_plan_t p, int32_t M, int32_t K, int64_t B,
                                               const void* H, const float* t, int64_t t_stride,
                                               const float* step, const float* lam, float a,
                                               float* loss, float* dstep, float* dlam,
                                               int32_t* flags, precode_stream_t stream) {
  return train_step_impl(p, M, K, B, H, t, t_stride, step, lam, a, nullptr, loss, dstep, dlam,
                         flags, stream);
}

extern "C" precode_status_t precode_train_step_supervised(
    precode_plan_t p, int32_t M, int32_t K, int64_t B, const void* H, const float* t,
    int64_t t_stride, const void* W_gt, const float* step, const float* lam, float* loss,
    float* dstep, float* dlam, int32_t* flags, precode_stream_t stream) {
  if (!W_gt) return fail(PRECODE_EINVAL, "precode_train_step_supervised: NULL W_gt");
  return train_step_impl(p, M, K, B, H, t, t_stride, step, lam, 0.f, W_gt, loss, dstep, dlam,
                         flags, stream);
}
