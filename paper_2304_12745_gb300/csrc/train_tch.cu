// Instantiation of the split-FP16 tensor-core training kernel (projected layer,
// K = 8, M = 64).
#include "registry.h"
#include "train_tch.cuh"

namespace precode {

// 3 blocks per SM: 165 registers without spills (the 2-block build takes 237).  On the
// 8,192-instance training step it is 5 % faster (more warps for a short persistent
// loop); on 65,536 resident instances 4 % slower.
void register_train_tch(std::vector<TrainVariant>& v) {
  TrainVariant x{kModeProj, 8, 64, true, (const void*)&train_tch_kernel<4, 3>,
                 TrainTCH<4>::SMEM_BYTES, 4 * 32, 4, true, true};
  x.cp_onchip = TrainTCH<4>::CP_ONCHIP;
  v.push_back(x);
}

}  // namespace precode
