// Launch arguments shared by the host dispatch and the device kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "precode.h"

namespace precode {

// One instance of an uneven batch: offsets in elements (complex for H/W, float for t).
struct InstDesc {
  int64_t h_off;
  int64_t w_off;
  int64_t t_off;
  int32_t M;
  int32_t K;
};
static_assert(sizeof(InstDesc) == sizeof(precode_inst_t), "descriptor layout matches the ABI");

// Default FP64-path threshold on the equilibrated Gram condition estimate
// max(d) / min(d).  The FP32 setup's error grows like (a few) x 2^-24 x that
// estimate; at 16 the FP32 path stays well inside 1e-4 (W) and 1e-5 (objective)
// of the FP64 oracle on every kernel family, and everything above takes the FP64
// path (Gram factorised in FP64, layers in an orthonormal basis of the channel's
// row space), whose error does not grow with the conditioning.
constexpr float kDefaultCondThreshold = 16.f;

enum : uint32_t {
  OPT_STEP_NORMALISED = 1u,  // PGD: eta_l / (max_k sum_j |G_kj|)
  OPT_STALL_COPY = 2u,       // test aid: issue no channel copy, so every copy wait runs out
  OPT_FAC_EXPORT = 4u,       // write each instance's Gram factor into its slot of fac
};

// Resident Gram factor of one instance, in float2 units: the kernel's own
// G'^{-T} = (D H H^H D)^{-T} [KB][KB] (D its per-user power-of-two scales) and
// one entry whose x is 1 when that inverse is the FP32 path's (0: the instance
// takes the FP64 path and is set up in full every time).
__host__ __device__ constexpr int fac_stride(int KB) { return KB * KB + 2; }

struct SolveArgs {
  const float2* H;   // channel base
  const float* t;    // targets base
  int64_t t_stride;  // uniform batch: floats between instances' targets (0 = shared)
  const float* step; // [T] eta (PGD) or mu (PROJ)
  const float* lam;  // [T] lambda (PGD)
  float2* W;
  float* obj;
  float* resid;
  int32_t* flags;
  int64_t B;         // uniform batch size (ignored when tbl != nullptr)
  int32_t K, M, T;   // uniform shape
  float cond_thr;
  uint32_t opts;
  const InstDesc* tbl;    // uneven batch table (device), nullptr for uniform
  const int32_t* index;   // this bucket's instance ids (device)
  const int32_t* count;   // this bucket's instance count (device)
  unsigned long long* err;  // device counter of wait timeouts
  uint64_t wait_ns;         // limit of one channel-copy wait (0: the default, 1 s)
  float2* fac;              // resident Gram factors (kernels with Variant::fac), or nullptr
  const int64_t* fidx;      // per instance: its factor slot's offset in fac (float2), -1 none;
                            // with OPT_FAC_EXPORT the slot of instance i is fac + i fac_stride(KB)
};

}  // namespace precode
