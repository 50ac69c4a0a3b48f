// Instantiations of the multi-warp tensor-core (split TF32) solve kernel for
// 128 antennas: exact builds serve their bucket shape, padded builds any K <= KB
// users at exactly 128 antennas.
#include "registry.h"
#include "solve_tcw.cuh"

namespace precode {

void register_solve_tcw_128(std::vector<Variant>& v) {
#define X(MODE, KW, MINB, EXACT)                                                             \
  v.push_back(Variant{MODE, 8 * KW, 128, KW, 8, 8, KW, MINB, EXACT, true, false,              \
                      (const void*)&solve_tcw_kernel<MODE, KW, 128, MINB>,                    \
                      TcwCfg<KW, 128>::SMEM_BYTES, KW * 32, 1, true});
  X(kModeProj, 2, 6, true)
  X(kModeProj, 2, 6, false)
  X(kModeProj, 1, 12, false)
  X(kModeProj, 3, 4, false)
  X(kModeProj, 4, 3, false)
  X(kModePGD, 2, 6, true)
#undef X
}

}  // namespace precode
