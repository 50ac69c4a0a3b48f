// Instantiations of the multi-warp split-FP16 projected-layer kernel: exact
// builds serve their bucket shape, padded builds any K <= KB users at exactly MB
// antennas.
#include "registry.h"
#include "solve_tcwh.cuh"

namespace precode {

void register_solve_tcwh(std::vector<Variant>& v) {
#define X(KW, MB, MINB, EXACT)                                                             \
  {                                                                                        \
    Variant x{kModeProj, 8 * KW, MB, KW, 8, 8, KW, MINB, EXACT, true, false,               \
              (const void*)&solve_tcwh_kernel<KW, MB, MINB>, TcwhCfg<KW, MB>::SMEM_BYTES,  \
              KW * 32, 1, true, true};                                                     \
    x.fac = true;                                                                          \
    v.push_back(x);                                                                        \
  }
  X(4, 256, 2, true)
  X(4, 256, 2, false)
  X(3, 256, 2, false)
  X(2, 256, 4, false)
  X(2, 128, 6, true)
  X(2, 128, 6, false)
  X(3, 128, 4, false)
  X(4, 128, 3, false)
  X(2, 64, 8, false)
  X(3, 64, 5, false)
  X(4, 64, 4, false)
#undef X
}

}  // namespace precode
