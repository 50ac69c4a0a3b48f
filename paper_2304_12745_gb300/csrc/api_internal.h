// Internal helpers shared by the host-side translation units.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "kernel_args.h"
#include "precode.h"
#include "registry.h"

namespace precode {

precode_status_t fail(precode_status_t st, const std::string& msg);
precode_status_t cuda_fail(cudaError_t e, const char* what);

// Every device and page-locked host allocation of the library goes through these
// two.  Test aid: with PRECODE_INJECT_ENOMEM=N (N >= 1) in the environment, the
// N-th allocation counted from the moment the variable took its current value
// fails with cudaErrorMemoryAllocation without reaching the CUDA allocator.
cudaError_t dev_alloc(void** ptr, size_t bytes);
cudaError_t pinned_alloc(void** ptr, size_t bytes);
template <class T>
cudaError_t dev_alloc(T** ptr, size_t bytes) {
  return dev_alloc(reinterpret_cast<void**>(ptr), bytes);
}
template <class T>
cudaError_t pinned_alloc(T** ptr, size_t bytes) {
  return pinned_alloc(reinterpret_cast<void**>(ptr), bytes);
}

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev);
  ~DeviceGuard();

 private:
  int prev_ = 0;
};

bool shape_ok(int mode, int M, int K);
// (Re)build plan->buckets from plan->shapes / plan->chosen plus one generic bucket
// per bucket size, so every shape a plan bucket can hold has a home.
void plan_build_buckets(precode_plan_t p);
int variant_occupancy(const Variant& v, int device);
// Default variant for (mode, M, K): the tensor-core build if requested and present,
// else the first exact build, else the smallest generic bucket holding the shape.
const Variant* pick_variant(int mode, int M, int K, bool tensor_cores = false);
// Allocates the plan's uneven-batch workspace (bucket lists) if not yet there.
precode_status_t ensure_workspace(precode_plan_t p);
std::vector<const Variant*> eligible_variants(int mode, int M, int K);
// n_hint >= 0: launch no more blocks than needed for n_hint instances.
precode_status_t launch_variant(const Variant& v, int device, int num_sms, const SolveArgs& A,
                                int64_t n_hint, cudaStream_t stream);

// One bucket of an uneven batch: instances of exactly (M, K) when the variant is an
// exact build, else every shape the generic variant holds.
struct Bucket {
  int M, K;
  const Variant* v;
};

// precode_solve_varlen with resident Gram factors: fidx[b] >= 0 is the float2
// offset in fac of instance b's factor slot (nullptr fac / fidx: none).  bucket_n
// (host, one count per plan bucket as bucket_of assigns them, or nullptr): empty
// buckets launch nothing and the others no more blocks than they need (ignored
// with PRECODE_PLAN_GRAPHS).
precode_status_t solve_varlen_fac(precode_plan_t p, int64_t B, const precode_inst_t* tbl,
                                  const void* H, const float* t, const float* step,
                                  const float* lam, void* W, float* obj, float* resid,
                                  int32_t* flags, float2* fac, const int64_t* fidx,
                                  precode_stream_t stream, const int64_t* bucket_n);
// The plan bucket the device bucketing assigns to a valid (M, K), or -1.
int bucket_of(precode_plan_t p, int M, int K);

// Resident Gram factors of n instances of shape (M, K) (device H [n][K][M], scratch
// W of the same size, t: K device floats), computed by the kernel the plan runs for
// that shape and written to fac, slot i at i * (*stride) float2.  *stride = 0 when
// that kernel does not keep factors (nothing is launched then).
precode_status_t plan_export_factors(precode_plan_t p, int32_t M, int32_t K, int64_t n,
                                     const void* H, float2* fac, void* W, const float* t,
                                     cudaStream_t stream, int* stride);

}  // namespace precode

struct precode_plan_s {
  int mode = 0, T = 0, device = 0, num_sms = 0;
  std::vector<precode_shape_t> shapes;
  std::vector<const precode::Variant*> chosen;
  // uneven batches: buckets, instance lists, counts and the captured graph
  std::vector<precode::Bucket> buckets;
  int32_t* d_index = nullptr;  // [n_buckets][max_instances]
  int32_t* d_count = nullptr;  // [n_buckets]
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<cudaGraphNode_t> graph_nodes;  // bucketize, then one solve node per bucket
  // training: checkpoints and per-instance loss / gradient partials
  float2* d_cp = nullptr;
  size_t cp_bytes = 0;
  float* d_part = nullptr;
  size_t part_bytes = 0;

  int64_t max_instances = 0;
  float cond_thr = 1e3f;
  uint32_t flags = 0;
  unsigned long long* d_err = nullptr;
  // host-buffer pipeline
  static constexpr int kPipe = 4;
  cudaStream_t hstream[kPipe] = {};
  int64_t chunk = 0;
  size_t chunk_elems = 0;  // complex elements per chunk buffer
  void* dH[kPipe] = {};
  void* dW[kPipe] = {};
  // whole-batch targets and per-instance outputs (one copy each way per call)
  int64_t out_cap = 0, t_cap = 0;
  float* dt_all = nullptr;
  float* dobj_all = nullptr;
  float* dres_all = nullptr;
  int32_t* dfl_all = nullptr;
  cudaEvent_t hev[kPipe + 1] = {};
  float* dparams = nullptr;  // [2][T]
  std::mutex mu;
  // test aid (precode_plan_set_debug): limit of the kernels' channel-copy waits
  // (0 = the default) and copy-stall injection
  uint64_t wait_ns = 0;
  bool stall_copy = false;

  // Kernel option bits of this plan's launches.
  uint32_t kernel_opts() const {
    return ((flags & PRECODE_PLAN_STEP_NORMALISED) ? precode::OPT_STEP_NORMALISED : 0u) |
           (stall_copy ? precode::OPT_STALL_COPY : 0u);
  }

  // Variant serving (M, K): the plan shape's own variant, else the smallest
  // generic bucket of the plan that holds the shape (nullptr if none).
  const precode::Variant* variant_for(int M, int K) const {
    for (size_t i = 0; i < shapes.size(); ++i)
      if (shapes[i].M == M && shapes[i].K == K) return chosen[i];
    // smallest bucket that fits; on a tie the tensor-core build (as bucketize_kernel)
    const precode::Variant* best = nullptr;
    auto score = [](const precode::Variant* v) { return 2 * v->KB * v->MB - (v->tc ? 1 : 0); };
    for (const auto& bk : buckets) {
      const precode::Variant* v = bk.v;
      if (!v->exact && precode::variant_fits(*v, M, K) && (!best || score(v) < score(best))) best = v;
    }
    return best;
  }
};


