// Instantiations of the split-FP16 tensor-core solve kernel (K = 8, M = 64):
// the projected layer and the paper layer.
#include "registry.h"
#include "solve_tch.cuh"

namespace precode {

void register_solve_tch(std::vector<Variant>& v) {
#define X(NW, MINB)                                                                     \
  {                                                                                     \
    Variant x{kModeProj, 8, 64, 4, 8, 8, NW, MINB, true, true, false,                   \
              (const void*)&solve_tch_kernel<NW, MINB>, SolveTCH<NW>::SMEM_BYTES,       \
              NW * 32, NW, true, true};                                                 \
    x.fac = true;                                                                       \
    v.push_back(x);                                                                     \
  }
  X(4, 3)
  X(4, 4)
#undef X
  // the paper layer (one global scale on the channel): 126 registers, 4 blocks per SM
  // (held to 3 by a larger shared-memory request it ran 3 % slower)
  v.push_back(Variant{kModePGD, 8, 64, 4, 8, 8, 4, 4, true, true, false,
                      (const void*)&solve_tch_kernel<4, 4, false, kModePGD>,
                      SolveTCH<4, false, kModePGD>::SMEM_BYTES, 4 * 32, 4, true, true});
}

// The same builds reading H, t and writing W and the outputs with plain loads and
// stores, for page-locked host buffers mapped into the device's address space.
const void* tch_host_kernel(int nw, int minb) {
  if (nw == 4 && minb == 3) return (const void*)&solve_tch_kernel<4, 3, true>;
  if (nw == 4 && minb == 4) return (const void*)&solve_tch_kernel<4, 4, true>;
  return nullptr;
}

}  // namespace precode
