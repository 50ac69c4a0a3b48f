// Instantiations of the multi-warp tensor-core (split TF32) solve kernel for
// 64 antennas: exact builds serve their bucket shape, padded builds any K <= KB
// users at exactly 64 antennas.
#include "registry.h"
#include "solve_tcw.cuh"

namespace precode {

void register_solve_tcw_64(std::vector<Variant>& v) {
#define X(MODE, KW, MINB, EXACT)                                                             \
  v.push_back(Variant{MODE, 8 * KW, 64, KW, 8, 8, KW, MINB, EXACT, true, false,              \
                      (const void*)&solve_tcw_kernel<MODE, KW, 64, MINB>,                    \
                      TcwCfg<KW, 64>::SMEM_BYTES, KW * 32, 1, true});
  X(kModeProj, 1, 16, false)
  X(kModeProj, 2, 8, false)
  X(kModeProj, 3, 5, false)
  X(kModeProj, 4, 4, false)
#undef X
}

}  // namespace precode
