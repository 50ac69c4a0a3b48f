// Instantiation of the transposed tcgen05 projected-layer kernel: any K <= 32
// users at exactly 256 antennas (users padded to 32).
#include "registry.h"
#include "solve_tgt.cuh"

namespace precode {

void register_solve_tgt(std::vector<Variant>& v) {
  Variant x{kModeProj, 32, 256, 4, 8, 8, TgCfg::NT / 32, 1, false, true, false,
            (const void*)&solve_tgt_kernel, TgCfg::SMEM_BYTES, TgCfg::NT, 1, true, true};
  x.tg = true;
  x.fac = true;
  x.tgt = true;
  v.push_back(x);
}

}  // namespace precode
