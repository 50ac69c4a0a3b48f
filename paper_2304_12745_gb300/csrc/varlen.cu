// Uneven batches: a device-side bucketing kernel assigns every instance
// descriptor to a plan bucket (counting sort with per-bucket atomic counters),
// then one persistent solve launch per bucket walks that bucket's instance list.
// With PRECODE_PLAN_GRAPHS the memset, the bucketing kernel and the per-bucket
// solves form one CUDA graph (the solves are parallel branches); each call only
// rewrites the kernel-node arguments and launches the graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "api_internal.h"

namespace precode {

namespace {

constexpr int kMaxBuckets = 32;

struct BucketTable {
  int n;
  int mode;
  int M[kMaxBuckets], K[kMaxBuckets], KB[kMaxBuckets], MB[kMaxBuckets], exact[kMaxBuckets];
  int mfix[kMaxBuckets];  // non-exact bucket that needs M == MB (user-padded tensor-core build)
};

__global__ void bucketize_kernel(const InstDesc* __restrict__ tbl, int64_t B, BucketTable bt,
                                 int32_t* __restrict__ index, int64_t stride,
                                 int32_t* __restrict__ count, int32_t* __restrict__ flags) {
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < B;
       b += (int64_t)gridDim.x * blockDim.x) {
    const InstDesc d = tbl[b];
    bool ok = d.K >= 1 && d.K <= PRECODE_MAX_K && d.M >= 2 && d.M <= PRECODE_MAX_M &&
              (d.M & 1) == 0 && (bt.mode != PRECODE_LAYER_PROJ || d.K <= d.M) && d.h_off >= 0 &&
              d.w_off >= 0 && d.t_off >= 0 && (d.h_off & 1) == 0 && (d.w_off & 1) == 0;
    int s = -1;
    if (ok) {
      for (int i = 0; i < bt.n; ++i)
        if (bt.exact[i] && bt.M[i] == d.M && bt.K[i] == d.K) s = i;
      if (s < 0) {
        int best = 1 << 30;
        for (int i = 0; i < bt.n; ++i)
          // smallest bucket; on a tie the tensor-core build (as the host's variant_for)
          if (!bt.exact[i] && bt.KB[i] >= d.K && bt.MB[i] >= d.M && (!bt.mfix[i] || bt.MB[i] == d.M) &&
              2 * bt.KB[i] * bt.MB[i] - bt.mfix[i] < best) {
            best = 2 * bt.KB[i] * bt.MB[i] - bt.mfix[i];
            s = i;
          }
      }
    }
    if (s < 0) {
      if (flags) flags[b] = PRECODE_F_INVALID;
      continue;
    }
    const int pos = atomicAdd(count + s, 1);
    index[s * stride + pos] = (int32_t)b;
  }
}

struct VarlenCall {
  BucketTable bt;
  std::vector<SolveArgs> args;  // per bucket
  const InstDesc* tbl;
  int64_t B;
  int32_t* flags;
};

}  // namespace

// The bucket bucketize_kernel assigns to a valid (M, K) on this plan, on the host
// (the same rule: the exact bucket of the shape, else the smallest generic bucket
// that holds it, a tensor-core build that needs M == MB winning ties); -1 if none.
int bucket_of(precode_plan_t p, int M, int K) {
  const int nb = (int)p->buckets.size();
  for (int i = 0; i < nb; ++i) {
    const Variant* v = p->buckets[i].v;
    if (v->exact && p->buckets[i].M == M && p->buckets[i].K == K) return i;
  }
  int s = -1, best = 1 << 30;
  for (int i = 0; i < nb; ++i) {
    const Variant* v = p->buckets[i].v;
    const int mfix = (!v->exact && v->tc) ? 1 : 0;
    if (!v->exact && v->KB >= K && v->MB >= M && (!mfix || v->MB == M) &&
        2 * v->KB * v->MB - mfix < best) {
      best = 2 * v->KB * v->MB - mfix;
      s = i;
    }
  }
  return s;
}

precode_status_t ensure_workspace(precode_plan_t p) {
  if (p->d_index) return PRECODE_OK;
  const size_t nb = p->buckets.size();
  if (dev_alloc(&p->d_index, sizeof(int32_t) * nb * (size_t)p->max_instances) != cudaSuccess ||
      dev_alloc(&p->d_count, sizeof(int32_t) * nb) != cudaSuccess) {
    cudaFree(p->d_index);
    p->d_index = nullptr;
    return fail(PRECODE_ENOMEM, "precode_solve_varlen: bucket workspace");
  }
  return PRECODE_OK;
}

namespace {

int bucketize_grid(precode_plan_t p) { return 2 * p->num_sms; }

void fill_args(precode_plan_t p, VarlenCall& call, const precode_inst_t* tbl, int64_t B,
               const void* H, const float* t, const float* step, const float* lam, void* W,
               float* obj, float* resid, int32_t* flags, float2* fac = nullptr,
               const int64_t* fidx = nullptr) {
  const int nb = (int)p->buckets.size();
  call.bt.n = nb;
  call.bt.mode = p->mode;
  for (int i = 0; i < nb; ++i) {
    const Variant* v = p->buckets[i].v;
    call.bt.M[i] = p->buckets[i].M;
    call.bt.K[i] = p->buckets[i].K;
    call.bt.KB[i] = v->KB;
    call.bt.MB[i] = v->MB;
    call.bt.exact[i] = v->exact ? 1 : 0;
    call.bt.mfix[i] = (!v->exact && v->tc) ? 1 : 0;
  }
  call.tbl = reinterpret_cast<const InstDesc*>(tbl);
  call.B = B;
  call.flags = flags;
  call.args.assign(nb, SolveArgs{});
  for (int i = 0; i < nb; ++i) {
    SolveArgs& A = call.args[i];
    A.H = static_cast<const float2*>(H);
    A.t = t;
    A.t_stride = 0;
    A.step = step;
    A.lam = lam ? lam : step;
    A.W = static_cast<float2*>(W);
    A.obj = obj;
    A.resid = resid;
    A.flags = flags;
    A.B = 0;
    A.K = p->buckets[i].K;
    A.M = p->buckets[i].M;
    A.T = p->T;
    A.cond_thr = p->cond_thr;
    A.opts = p->kernel_opts();
    A.wait_ns = p->wait_ns;
    A.tbl = call.tbl;
    A.fac = p->buckets[i].v->fac ? fac : nullptr;
    A.fidx = p->buckets[i].v->fac ? fidx : nullptr;
    A.index = p->d_index + (size_t)i * p->max_instances;
    A.count = p->d_count + i;
    A.err = p->d_err;
  }
}

precode_status_t build_graph(precode_plan_t p, VarlenCall& call) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return cuda_fail(e, "varlen graph create");
  const int nb = (int)p->buckets.size();
  cudaMemsetParams ms{};
  ms.dst = p->d_count;
  ms.value = 0;
  ms.elementSize = 4;
  ms.width = nb;
  ms.height = 1;
  cudaGraphNode_t memset_node, bucket_node;
  e = cudaGraphAddMemsetNode(&memset_node, g, nullptr, 0, &ms);
  std::vector<cudaGraphNode_t> nodes;
  if (e == cudaSuccess) {
    int64_t stride = p->max_instances;
    void* kargs[] = {(void*)&call.tbl, (void*)&call.B, (void*)&call.bt, (void*)&p->d_index,
                     (void*)&stride, (void*)&p->d_count, (void*)&call.flags};
    cudaKernelNodeParams kp{};
    kp.func = (void*)bucketize_kernel;
    kp.gridDim = dim3(bucketize_grid(p));
    kp.blockDim = dim3(256);
    kp.kernelParams = kargs;
    e = cudaGraphAddKernelNode(&bucket_node, g, &memset_node, 1, &kp);
    nodes.push_back(bucket_node);
  }
  for (int i = 0; i < nb && e == cudaSuccess; ++i) {
    const Variant* v = p->buckets[i].v;
    void* kargs[] = {(void*)&call.args[i]};
    cudaKernelNodeParams kp{};
    kp.func = (void*)v->fn;
    kp.gridDim = dim3(variant_occupancy(*v, p->device) * p->num_sms);
    kp.blockDim = dim3(v->threads);
    kp.sharedMemBytes = v->smem;
    kp.kernelParams = kargs;
    cudaGraphNode_t n;
    e = cudaGraphAddKernelNode(&n, g, &bucket_node, 1, &kp);
    nodes.push_back(n);
  }
  cudaGraphExec_t ex = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ex, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "varlen graph build");
  }
  p->graph = g;
  p->graph_exec = ex;
  p->graph_nodes = nodes;
  return PRECODE_OK;
}

precode_status_t update_graph(precode_plan_t p, VarlenCall& call) {
  int64_t stride = p->max_instances;
  void* kargs[] = {(void*)&call.tbl, (void*)&call.B, (void*)&call.bt, (void*)&p->d_index,
                   (void*)&stride, (void*)&p->d_count, (void*)&call.flags};
  cudaKernelNodeParams kp{};
  kp.func = (void*)bucketize_kernel;
  kp.gridDim = dim3(bucketize_grid(p));
  kp.blockDim = dim3(256);
  kp.kernelParams = kargs;
  cudaError_t e = cudaGraphExecKernelNodeSetParams(p->graph_exec, p->graph_nodes[0], &kp);
  for (size_t i = 0; i < p->buckets.size() && e == cudaSuccess; ++i) {
    const Variant* v = p->buckets[i].v;
    void* sargs[] = {(void*)&call.args[i]};
    cudaKernelNodeParams sp{};
    sp.func = (void*)v->fn;
    sp.gridDim = dim3(variant_occupancy(*v, p->device) * p->num_sms);
    sp.blockDim = dim3(v->threads);
    sp.sharedMemBytes = v->smem;
    sp.kernelParams = sargs;
    e = cudaGraphExecKernelNodeSetParams(p->graph_exec, p->graph_nodes[i + 1], &sp);
  }
  if (e != cudaSuccess) return cuda_fail(e, "varlen graph update");
  return PRECODE_OK;
}

}  // namespace

}  // namespace precode

using namespace precode;

extern "C" precode_status_t precode_solve_varlen(precode_plan_t p, int64_t B,
                                                 const precode_inst_t* tbl, const void* H,
                                                 const float* t, const float* step,
                                                 const float* lam, void* W, float* obj,
                                                 float* resid, int32_t* flags,
                                                 precode_stream_t stream) {
  return precode::solve_varlen_fac(p, B, tbl, H, t, step, lam, W, obj, resid, flags, nullptr,
                                   nullptr, stream, nullptr);
}

// The uneven-batch solve with optional resident Gram factors: fidx[b] >= 0 names
// instance b's factor slot in fac (float2 offset), for the buckets whose kernel
// imports them.
precode_status_t precode::solve_varlen_fac(precode_plan_t p, int64_t B, const precode_inst_t* tbl,
                                           const void* H, const float* t, const float* step,
                                           const float* lam, void* W, float* obj, float* resid,
                                           int32_t* flags, float2* fac, const int64_t* fidx,
                                           precode_stream_t stream, const int64_t* bucket_n) {
  if (!p) return fail(PRECODE_EINVAL, "precode_solve_varlen: NULL plan");
  if (B < 0 || B > p->max_instances)
    return fail(PRECODE_EINVAL, "precode_solve_varlen: B outside [0, max_instances]");
  if (B == 0) return PRECODE_OK;
  if (!tbl || !H || !t || !step || !W) return fail(PRECODE_EINVAL, "precode_solve_varlen: NULL buffer");
  if (p->mode == PRECODE_LAYER_PGD && !lam)
    return fail(PRECODE_EINVAL, "precode_solve_varlen: lam required for the paper layer");
  if (((uintptr_t)H & 15) || ((uintptr_t)W & 15) || ((uintptr_t)tbl & 7))
    return fail(PRECODE_EINVAL, "precode_solve_varlen: misaligned buffer");
  if ((int)p->buckets.size() > kMaxBuckets)
    return fail(PRECODE_EINVAL, "precode_solve_varlen: plan has too many buckets");
  std::lock_guard<std::mutex> lk(p->mu);
  DeviceGuard g(p->device);
  precode_status_t st = ensure_workspace(p);
  if (st != PRECODE_OK) return st;
  VarlenCall call;
  fill_args(p, call, tbl, B, H, t, step, lam, W, obj, resid, flags, fac, fidx);
  cudaStream_t s = (cudaStream_t)stream;
  if (p->flags & PRECODE_PLAN_GRAPHS) {
    if (!p->graph_exec) {
      st = build_graph(p, call);
      if (st != PRECODE_OK) return st;
    } else {
      st = update_graph(p, call);
      if (st != PRECODE_OK) return st;
    }
    cudaError_t e = cudaGraphLaunch(p->graph_exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "precode_solve_varlen: graph launch");
    return PRECODE_OK;
  }
  cudaError_t e = cudaMemsetAsync(p->d_count, 0, sizeof(int32_t) * p->buckets.size(), s);
  if (e != cudaSuccess) return cuda_fail(e, "precode_solve_varlen: memset");
  bucketize_kernel<<<bucketize_grid(p), 256, 0, s>>>(call.tbl, B, call.bt, p->d_index,
                                                      p->max_instances, p->d_count, flags);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "precode_solve_varlen: bucketize launch");
  for (size_t i = 0; i < p->buckets.size(); ++i) {
    // with the buckets' instance counts known on the host: no launch for an empty
    // bucket, and no more blocks than its instances need
    if (bucket_n && bucket_n[i] == 0) continue;
    st = launch_variant(*p->buckets[i].v, p->device, p->num_sms, call.args[i],
                        bucket_n ? bucket_n[i] : -1, s);
    if (st != PRECODE_OK) return st;
  }
  return PRECODE_OK;
}
