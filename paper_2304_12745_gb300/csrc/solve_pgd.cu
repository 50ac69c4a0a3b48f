// Instantiations of the solve kernel for the paper layer (Sec. V, Eq. unfoldednet).
#include "registry.h"
#include "solve.cuh"

namespace precode {

void register_solve_pgd(std::vector<Variant>& v) {
#define X(KB, MB, GK, GM, JC, EXACT, NW, MINB, SPLIT, DB)                                                 \
  v.push_back(Variant{kModePGD, KB, MB, GK, GM, JC, NW, MINB, EXACT, SPLIT, DB,                           \
                      (const void*)&solve_kernel<kModePGD, KB, MB, GK, GM, JC, EXACT, NW, MINB, SPLIT, DB>, \
                      SolveCfg<kModePGD, KB, MB, GK, GM, JC, NW, DB>::SMEM_BYTES, NW * 32,      \
                      SolveCfg<kModePGD, KB, MB, GK, GM, JC, NW, DB>::GROUPS, false});
#include "solve_variants.inc"
#undef X
}

}  // namespace precode
