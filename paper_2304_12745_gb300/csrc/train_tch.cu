// Instantiation of the split-FP16 tensor-core training kernel (projected layer,
// K = 8, M = 64).
#include "registry.h"
#include "train_tch.cuh"

namespace precode {

// One block of 12 warps per SM (a tensor-memory kernel is resident once per SM): the
// warps of three 4-warp blocks, at the register budget of the 3-block build (under 168
// registers, no spills).
void register_train_tch(std::vector<TrainVariant>& v) {
  TrainVariant x{kModeProj, 8, 64, true, (const void*)&train_tch_kernel<12, 1>,
                 TrainTCH<12>::SMEM_BYTES, 12 * 32, 12, true, true};
  x.cp_onchip = TrainTCH<12>::CP_ONCHIP;
  v.push_back(x);
}

}  // namespace precode
