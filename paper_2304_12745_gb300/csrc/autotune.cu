// Autotuner: for every shape of a plan, time each compiled kernel variant that
// can serve it on synthetic channels and keep the fastest.  Results are cached
// in a text file keyed by device name, mode, K and M, so later plans skip the
// timing.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>

#include "api_internal.h"

namespace precode {

namespace {

// Deterministic pseudo-random CN(0,1)-like entries for timing only.
__global__ void fill_timing_channels(float2* H, int64_t n, uint32_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t x = (uint32_t)i * 2654435761u ^ seed;
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    const float u1 = ((x & 0xffff) + 0.5f) / 65536.f, u2 = ((x >> 16) + 0.5f) / 65536.f;
    H[i] = make_float2(u1 - 0.5f, u2 - 0.5f);
  }
}

__global__ void fill_const(float* p, int64_t n, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

std::string variant_key(const Variant& v) {
  std::ostringstream o;
  o << v.KB << "x" << v.MB << "/" << v.GK << "x" << v.GM << "/jc" << v.JC << "/w" << v.NW
    << "/b" << v.minb << (v.split ? "/split" : "") << (v.tc ? "/tc" : "") << (v.f16 ? "/f16" : "") << (v.tg ? "/tg" : "") << (v.tgt ? "/tgt" : "") << (v.db ? "/db" : "") << (v.exact ? "/exact" : "/generic");
  return o.str();
}

}  // namespace

precode_status_t autotune_plan(precode_plan_t p, const char* cache_path) {
  const int dev = p->device;
  cudaDeviceProp prop{};
  cudaGetDeviceProperties(&prop, dev);
  std::map<std::string, std::string> cache;  // "dev|mode|K|M" -> variant key
  if (cache_path) {
    std::ifstream f(cache_path);
    std::string line;
    while (std::getline(f, line)) {
      const auto tab = line.find('\t');
      if (tab != std::string::npos) cache[line.substr(0, tab)] = line.substr(tab + 1);
    }
  }
  bool dirty = false;
  auto& shapes = p->shapes;
  auto& chosen = p->chosen;
  for (size_t si = 0; si < shapes.size(); ++si) {
    const int M = shapes[si].M, K = shapes[si].K;
    std::ostringstream ks;
    ks << prop.name << "|" << p->mode << "|" << K << "|" << M;
    const auto cands = eligible_variants(p->mode, M, K);
    auto hit = cache.find(ks.str());
    if (hit != cache.end()) {
      for (auto* v : cands)
        if (variant_key(*v) == hit->second && variant_occupancy(*v, dev) > 0) chosen[si] = v;
      continue;
    }
    const int64_t B = std::min<int64_t>(p->max_instances, 16384);
    const int T = p->T;
    float2 *H = nullptr, *W = nullptr;
    float *t = nullptr, *prm = nullptr;
    if (dev_alloc(&H, (size_t)B * K * M * 8) != cudaSuccess ||
        dev_alloc(&W, (size_t)B * K * M * 8) != cudaSuccess ||
        dev_alloc(&t, (size_t)K * 4) != cudaSuccess ||
        dev_alloc(&prm, (size_t)2 * T * 4) != cudaSuccess) {
      cudaFree(H);
      cudaFree(W);
      cudaFree(t);
      cudaFree(prm);
      return fail(PRECODE_ENOMEM, "autotune: timing buffers");
    }
    fill_timing_channels<<<256, 256>>>(H, (int64_t)B * K * M, 12345u);
    fill_const<<<1, 256>>>(t, K, 1.f);
    fill_const<<<1, 256>>>(prm, 2 * T, 0.01f);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    const Variant* best = chosen[si];
    for (auto* v : cands) {
      if (variant_occupancy(*v, dev) <= 0) continue;
      SolveArgs A{};
      A.H = H;
      A.t = t;
      A.t_stride = 0;
      A.step = prm;
      A.lam = prm + T;
      A.W = W;
      A.B = B;
      A.K = K;
      A.M = M;
      A.T = T;
      A.cond_thr = p->cond_thr;
      A.err = p->d_err;
      float ms_min = 1e30f;
      for (int rep = 0; rep < 4; ++rep) {
        cudaEventRecord(e0);
        if (launch_variant(*v, dev, p->num_sms, A, B, 0) != PRECODE_OK) break;
        cudaEventRecord(e1);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_min = std::min(ms_min, ms);
      }
      if (std::getenv("PRECODE_TUNE_LOG"))
        std::fprintf(stderr, "[precode autotune] mode %d K=%d M=%d %s: %.4f ms\n", p->mode, K,
                     M, variant_key(*v).c_str(), ms_min);
      if (ms_min < best_ms) {
        best_ms = ms_min;
        best = v;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(H);
    cudaFree(W);
    cudaFree(t);
    cudaFree(prm);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "autotune");
    chosen[si] = best;
    cache[ks.str()] = variant_key(*best);
    dirty = true;
  }
  if (cache_path && dirty) {
    std::ofstream f(cache_path, std::ios::trunc);
    for (auto& kv : cache) f << kv.first << "\t" << kv.second << "\n";
  }
  return PRECODE_OK;
}

}  // namespace precode
