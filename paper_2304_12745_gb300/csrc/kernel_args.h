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

enum : uint32_t {
  OPT_STEP_NORMALISED = 1u,  // PGD: eta_l / (max_k sum_j |G_kj|)
};

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
};

}  // namespace precode
