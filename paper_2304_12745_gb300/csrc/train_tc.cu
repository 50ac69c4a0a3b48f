// Instantiations of the tensor-core (split TF32) training kernel, K = 8, M = 64.
#include "registry.h"
#include "train_tc.cuh"

namespace precode {

void register_train_tc(std::vector<TrainVariant>& v) {
#define X(MODE, NW, MINB)                                                                     \
  v.push_back(TrainVariant{MODE, 8, 64, true, (const void*)&train_tc_kernel<MODE, NW, MINB>,  \
                           TrainTC<MODE, NW>::SMEM_BYTES, NW * 32, NW, true});
  X(kModeProj, 4, 2)
  X(kModePGD, 4, 2)
#undef X
}

}  // namespace precode
