// Instantiations of the multi-warp tensor-core (split TF32) solve kernel for
// 256 antennas: exact builds serve their bucket shape, padded builds any K <= KB
// users at exactly 256 antennas.
#include "registry.h"
#include "solve_tcw.cuh"

namespace precode {

void register_solve_tcw_256(std::vector<Variant>& v) {
#define X(MODE, KW, MINB, EXACT)                                                             \
  v.push_back(Variant{MODE, 8 * KW, 256, KW, 8, 8, KW, MINB, EXACT, true, false,              \
                      (const void*)&solve_tcw_kernel<MODE, KW, 256, MINB>,                    \
                      TcwCfg<KW, 256>::SMEM_BYTES, KW * 32, 1, true});
  X(kModeProj, 4, 2, true)
  X(kModeProj, 4, 2, false)
  X(kModeProj, 1, 8, false)
  X(kModeProj, 2, 4, false)
  X(kModeProj, 3, 2, false)
  X(kModePGD, 4, 2, true)
#undef X
}

}  // namespace precode
