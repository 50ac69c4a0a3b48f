// Instantiations of the multi-warp tensor-core (split TF32) solve kernel for the
// 16 x 128 and 32 x 256 buckets.
#include "registry.h"
#include "solve_tcw.cuh"

namespace precode {

void register_solve_tcw(std::vector<Variant>& v) {
#define X(MODE, KW, MINB)                                                                  \
  v.push_back(Variant{MODE, 8 * KW, 64 * KW, KW, 8, 8, KW, MINB, true, true, false,       \
                      (const void*)&solve_tcw_kernel<MODE, KW, MINB>, TcwCfg<KW>::SMEM_BYTES, \
                      KW * 32, 1, true});
  X(kModeProj, 2, 6)
  X(kModeProj, 2, 8)
  X(kModeProj, 4, 2)
  X(kModePGD, 2, 6)
  X(kModePGD, 2, 8)
  X(kModePGD, 4, 2)
#undef X
}

}  // namespace precode
