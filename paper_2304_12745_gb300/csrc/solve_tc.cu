// Instantiations of the tensor-core (warp MMA, split TF32) solve kernel, K = 8, M = 64.
#include "registry.h"
#include "solve_tc.cuh"

namespace precode {

void register_solve_tc(std::vector<Variant>& v) {
#define X(MODE, NW, MINB, DB)                                                           \
  v.push_back(Variant{MODE, 8, 64, 4, 8, 8, NW, MINB, true, true, DB,                   \
                      (const void*)&solve_tc_kernel<MODE, NW, MINB, DB>,                \
                      SolveTC<MODE, NW, DB>::SMEM_BYTES, NW * 32,                       \
                      SolveTC<MODE, NW, DB>::C::GROUPS, true});
  X(kModeProj, 4, 3, false)
  X(kModeProj, 4, 3, true)
  X(kModePGD, 4, 3, false)
  X(kModePGD, 4, 3, true)
#undef X
}

}  // namespace precode
