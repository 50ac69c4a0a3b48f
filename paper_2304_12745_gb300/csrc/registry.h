// Kernel variant table: one entry per compiled instantiation of the solve kernel.
#pragma once

#include <vector>

#include "kernel_args.h"

namespace precode {

struct Variant {
  int mode;      // 0 paper layer, 1 projected layer
  int KB, MB;    // bucket: users and antennas the register/shared layout is built for
  int GK, GM;    // thread grid per instance (user rows x antenna columns)
  int JC;        // residual columns per reduction pass
  int NW;        // warps per block
  int minb;      // blocks per SM the register budget is built for
  bool exact;    // compiled for K == KB and M == MB only
  bool split;    // complex registers as scalar pairs instead of float2
  bool db;       // two channel buffers (next copy issued one instance ahead)
  const void* fn;
  int smem;      // dynamic shared memory per block (bytes)
  int threads;   // threads per block
  int groups;    // instances resident per block
  bool tc;       // contractions on the tensor cores (warp MMA, split TF32); a non-exact
                 // tensor-core build pads users (K <= KB) but needs M == MB
  bool f16 = false;  // the layers' contractions as split-FP16 MMAs (scaled instances)
  bool tg = false;   // tcgen05 build: operands in shared memory, accumulators in tensor memory
  bool fac = false;  // exports / imports resident Gram factors (SolveArgs::fac)
  bool tgt = false;  // the transposed tcgen05 build (a thread per antenna, Q^T in tensor memory)
};

// The instance shapes (M, K) a variant solves.
inline bool variant_fits(const Variant& v, int M, int K) {
  if (v.exact) return v.KB == K && v.MB == M;
  if (v.tc) return v.KB >= K && v.MB == M;
  return v.KB >= K && v.MB >= M;
}

struct TrainVariant {
  int mode;
  int KB, MB;
  bool exact;
  const void* fn;
  int smem;
  int threads;
  int groups;
  bool tc;  // tensor-core (split TF32) build
  bool f16 = false;  // the layers' contractions as split-FP16 MMAs (scaled instances)
  int cp_onchip = 0;  // up to this many checkpoints per instance stay in tensor memory
};

void register_solve_pgd(std::vector<Variant>& v);
void register_train_pgd(std::vector<TrainVariant>& v);
void register_train_proj(std::vector<TrainVariant>& v);
void register_train_tc(std::vector<TrainVariant>& v);
void register_train_tch(std::vector<TrainVariant>& v);
const std::vector<TrainVariant>& train_variants();
void register_solve_proj(std::vector<Variant>& v);
void register_solve_tc(std::vector<Variant>& v);
void register_solve_tch(std::vector<Variant>& v);
void register_solve_tcwh(std::vector<Variant>& v);
void register_solve_tg(std::vector<Variant>& v);
void register_solve_tgt(std::vector<Variant>& v);
const void* tch_host_kernel(int nw, int minb);  // host-buffer twin of a split-FP16 K=8 build
void register_solve_tcw_64(std::vector<Variant>& v);
void register_solve_tcw_128(std::vector<Variant>& v);
void register_solve_tcw_256(std::vector<Variant>& v);
const std::vector<Variant>& variants();

}  // namespace precode
