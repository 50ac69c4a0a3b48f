// Train-kernel instantiations for the paper layer.
#include "registry.h"
#include "train.cuh"

namespace precode {

void register_train_pgd(std::vector<TrainVariant>& v) {
#define X(KB, MB, GK, GM, JC, EXACT, NW, MINB)                                                \
  v.push_back(TrainVariant{kModePGD, KB, MB, EXACT,                                          \
                           (const void*)&train_kernel<kModePGD, KB, MB, GK, GM, JC, EXACT, NW, MINB>, \
                           TrainKernel<kModePGD, KB, MB, GK, GM, JC, EXACT, NW>::SMEM_BYTES, NW * 32, \
                           SolveCfg<kModePGD, KB, MB, GK, GM, JC, NW>::GROUPS, false});
#include "train_variants.inc"
#undef X
}

}  // namespace precode
