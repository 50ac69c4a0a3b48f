// Instantiations of the solve kernel for the projected layer (shrink + projection onto H W^T = S).
#include "registry.h"
#include "solve.cuh"

namespace precode {

void register_solve_proj(std::vector<Variant>& v) {
#define X(KB, MB, GK, GM, JC, EXACT, NW, MINB, SPLIT, DB)                                                 \
  v.push_back(Variant{kModeProj, KB, MB, GK, GM, JC, NW, MINB, EXACT, SPLIT, DB,                           \
                      (const void*)&solve_kernel<kModeProj, KB, MB, GK, GM, JC, EXACT, NW, MINB, SPLIT, DB>, \
                      SolveCfg<kModeProj, KB, MB, GK, GM, JC, NW, DB>::SMEM_BYTES, NW * 32,      \
                      SolveCfg<kModeProj, KB, MB, GK, GM, JC, NW, DB>::GROUPS, false});
#include "solve_variants.inc"
#undef X
}

}  // namespace precode
