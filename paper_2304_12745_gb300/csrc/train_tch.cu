// Instantiation of the split-FP16 tensor-core training kernel (projected layer,
// K = 8, M = 64).
#include "registry.h"
#include "train_tch.cuh"

namespace precode {

void register_train_tch(std::vector<TrainVariant>& v) {
  v.push_back(TrainVariant{kModeProj, 8, 64, true, (const void*)&train_tch_kernel<4, 2>,
                           TrainTCH<4>::SMEM_BYTES, 4 * 32, 4, true, true});
}

}  // namespace precode
