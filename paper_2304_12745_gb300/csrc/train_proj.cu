// Train-kernel instantiations for the projected layer.
#include "registry.h"
#include "train.cuh"

namespace precode {

void register_train_proj(std::vector<TrainVariant>& v) {
#define X(KB, MB, GK, GM, JC, EXACT, NW, MINB)                                                \
  v.push_back(TrainVariant{kModeProj, KB, MB, EXACT,                                          \
                           (const void*)&train_kernel<kModeProj, KB, MB, GK, GM, JC, EXACT, NW, MINB>, \
                           TrainKernel<kModeProj, KB, MB, GK, GM, JC, EXACT, NW>::SMEM_BYTES, NW * 32, \
                           SolveCfg<kModeProj, KB, MB, GK, GM, JC, NW>::GROUPS, false});
#include "train_variants.inc"
#undef X
}

}  // namespace precode
