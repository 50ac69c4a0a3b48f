// Internal helpers shared by the host-side translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "kernel_args.h"
#include "precode.h"
#include "registry.h"

namespace precode {

precode_status_t fail(precode_status_t st, const std::string& msg);
precode_status_t cuda_fail(cudaError_t e, const char* what);

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev);
  ~DeviceGuard();

 private:
  int prev_ = 0;
};

bool shape_ok(int mode, int M, int K);
int variant_occupancy(const Variant& v, int device);
const Variant* pick_variant(int mode, int M, int K);
std::vector<const Variant*> eligible_variants(int mode, int M, int K);
// n_hint >= 0: launch no more blocks than needed for n_hint instances.
precode_status_t launch_variant(const Variant& v, int device, int num_sms, const SolveArgs& A,
                                int64_t n_hint, cudaStream_t stream);

int plan_mode(precode_plan_t p);
int plan_T(precode_plan_t p);
int plan_device(precode_plan_t p);
int plan_num_sms(precode_plan_t p);
float plan_cond(precode_plan_t p);
uint32_t plan_flags(precode_plan_t p);
unsigned long long* plan_err(precode_plan_t p);
int64_t plan_max_instances(precode_plan_t p);
std::vector<precode_shape_t>& plan_shapes(precode_plan_t p);
std::vector<const Variant*>& plan_chosen(precode_plan_t p);
const Variant* plan_variant_for(precode_plan_t p, int M, int K);

}  // namespace precode
