// Serving: continuous batching of precoding jobs.
//
// A job is n_sc independent narrowband subcarrier channels of one (M, K) with
// host buffers for H (or a resident channel), targets and results.  submit()
// queues it and returns a ticket.  A dispatcher thread admits queued jobs in
// arrival order while (a) a stream slot is free and (b) the job's buffers fit in
// the server's device arena (admission by free device memory); the jobs admitted
// together form one bucketed uneven-batch launch on that slot: host->device
// copies, precode_solve_varlen on the slot's plan, device->host copies, event.
// Jobs that arrive while other launches run are admitted as soon as a slot and
// memory free up, so their work overlaps on the device with the launches in
// flight.  One completion thread per slot waits for its event, stamps the jobs
// done, returns their memory and wakes the dispatcher and any waiters.
// Per-instance results do not depend on the other jobs of a launch (same kernel
// variant per shape, no cross-instance arithmetic).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "api_internal.h"

namespace precode {

namespace {

double now_us() {
  using namespace std::chrono;
  return duration<double, std::micro>(steady_clock::now().time_since_epoch()).count();
}

// First-fit sub-allocator over one device allocation, 256-byte granules.
class Arena {
 public:
  void init(size_t bytes) {
    free_.clear();
    size_ = bytes & ~size_t(255);
    free_[0] = size_;
    used_ = 0;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t start = it->first + bytes;
        free_.erase(it);
        if (rest) free_[start] = rest;
        used_ += bytes;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = (bytes + 255) & ~size_t(255);
    if (bytes == 0) bytes = 256;
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t used() const { return used_; }
  size_t size() const { return size_; }

 private:
  std::map<size_t, size_t> free_;
  size_t size_ = 0, used_ = 0;
};

struct Channel {
  int M, K, n_sc;
  size_t off, bytes;
  size_t fac_off = 0, fac_bytes = 0;  // resident Gram factors (fac_stride 0: none)
  int fac_stride = 0;                 // float2 per subcarrier's slot
};

struct Job {
  uint64_t ticket;
  precode_job_t d;
  int64_t n;  // instances
  size_t h_off = 0, h_bytes = 0, w_off = 0, w_bytes = 0, t_off = 0, t_bytes = 0;
  bool resident = false;
  size_t res_h_off = 0;
  size_t fac_off = 0;  // its channel's factor slots (fac_stride 0: none)
  int fac_stride = 0;
  double submit_us = 0, start_us = 0, done_us = 0;
  precode_status_t status = PRECODE_PENDING;
  int64_t first = 0;  // index of its first instance inside its launch
};

struct Slot {
  cudaStream_t stream = nullptr;
  precode_plan_t plan = nullptr;
  precode_inst_t* h_tbl = nullptr;  // pinned
  int64_t* h_fidx = nullptr;        // pinned: per instance its factor slot, -1 none
  int64_t* d_fidx = nullptr;
  // per-instance outputs of the launch, staged in pinned memory: a copy into a
  // caller's pageable buffer would hold the dispatcher until the launch ends
  float* h_obj = nullptr;
  float* h_resid = nullptr;
  int32_t* h_flags = nullptr;
  void* d_tbl = nullptr;
  float* d_obj = nullptr;
  float* d_resid = nullptr;
  int32_t* d_flags = nullptr;
  cudaEvent_t done = nullptr;
  std::vector<std::shared_ptr<Job>> jobs;
  bool busy = false;
  std::thread waiter;
  std::condition_variable cv;
  bool go = false;
};

}  // namespace

}  // namespace precode

using namespace precode;

struct precode_server_s {
  precode_serve_desc_t desc{};
  std::vector<precode_shape_t> shapes;
  int device = 0;
  void* arena_base = nullptr;
  Arena arena;
  float* d_step = nullptr;
  float* d_lam = nullptr;
  std::vector<std::unique_ptr<Slot>> slots;
  std::mutex mu;
  std::condition_variable cv_dispatch;  // new work or freed resources
  std::condition_variable cv_done;      // a job finished
  std::deque<std::shared_ptr<Job>> queue;
  std::unordered_map<uint64_t, std::shared_ptr<Job>> jobs;  // not yet retrieved
  std::unordered_map<uint64_t, Channel> channels;
  uint64_t next_ticket = 1, next_channel = 1;
  bool stop = false;
  std::thread dispatcher;
  // statistics
  uint64_t submitted = 0, completed = 0, rejected = 0, launches = 0;
  int64_t instances_done = 0, factor_instances = 0;
  double first_submit_us = 0, last_done_us = 0;
  std::vector<double> latencies;  // per completed job (us)
  std::string error;              // first asynchronous CUDA error
};

namespace precode {
namespace {

size_t job_t_floats(const precode_job_t& j) { return j.t_shared ? (size_t)j.K : (size_t)j.n_sc * j.K; }

// Dispatcher: admits jobs in arrival order into free slots.
void dispatch_loop(precode_server_t s) {
  DeviceGuard g(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    Slot* slot = nullptr;
    for (auto& sl : s->slots)
      if (!sl->busy) {
        slot = sl.get();
        break;
      }
    if (!slot || s->queue.empty()) {
      s->cv_dispatch.wait(lk);
      continue;
    }
    // form a launch from the head of the queue
    std::vector<std::shared_ptr<Job>> batch;
    int64_t n = 0;
    while (!s->queue.empty()) {
      auto& j = s->queue.front();
      if (n + j->n > s->desc.max_batch_instances && !batch.empty()) break;
      // admission by free arena memory
      bool ok = true;
      if (!j->resident && !s->arena.alloc(j->h_bytes, &j->h_off)) ok = false;
      if (ok && !s->arena.alloc(j->w_bytes, &j->w_off)) {
        if (!j->resident) s->arena.release(j->h_off, j->h_bytes);
        ok = false;
      }
      if (ok && !s->arena.alloc(j->t_bytes, &j->t_off)) {
        if (!j->resident) s->arena.release(j->h_off, j->h_bytes);
        s->arena.release(j->w_off, j->w_bytes);
        ok = false;
      }
      if (!ok) break;  // wait for memory; keep arrival order
      j->first = n;
      n += j->n;
      batch.push_back(j);
      s->queue.pop_front();
    }
    if (batch.empty()) {
      s->cv_dispatch.wait(lk);
      continue;
    }
    slot->busy = true;
    slot->jobs = batch;
    const double t_start = now_us();
    lk.unlock();
    // ---- issue the launch (no lock held)
    char* base = static_cast<char*>(s->arena_base);
    cudaStream_t st = slot->stream;
    cudaError_t e = cudaSuccess;
    int64_t b = 0, n_fac = 0;
    std::vector<int64_t> bucket_n(slot->plan->buckets.size(), 0);
    for (auto& j : batch) {
      j->start_us = t_start;
      const int bk = bucket_of(slot->plan, j->d.M, j->d.K);
      if (bk >= 0) bucket_n[bk] += j->n;
      const size_t hoff = j->resident ? j->res_h_off : j->h_off;
      if (!j->resident && e == cudaSuccess)
        e = cudaMemcpyAsync(base + hoff, j->d.H, j->h_bytes, cudaMemcpyHostToDevice, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + j->t_off, j->d.t, sizeof(float) * job_t_floats(j->d),
                            cudaMemcpyHostToDevice, st);
      const int64_t kk = j->d.K, mm = j->d.M;
      for (int64_t i = 0; i < j->n; ++i, ++b) {
        precode_inst_t& d = slot->h_tbl[b];
        d.h_off = (int64_t)(hoff / 8) + i * kk * mm;
        d.w_off = (int64_t)(j->w_off / 8) + i * kk * mm;
        d.t_off = (int64_t)(j->t_off / 4) + (j->d.t_shared ? 0 : i * kk);
        d.M = (int32_t)mm;
        d.K = (int32_t)kk;
        slot->h_fidx[b] = j->fac_stride ? (int64_t)(j->fac_off / 8) + i * j->fac_stride : -1;
        n_fac += j->fac_stride ? 1 : 0;
      }
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(slot->d_tbl, slot->h_tbl, sizeof(precode_inst_t) * n,
                          cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_fac)
      e = cudaMemcpyAsync(slot->d_fidx, slot->h_fidx, sizeof(int64_t) * n, cudaMemcpyHostToDevice, st);
    precode_status_t ps = PRECODE_OK;
    if (e == cudaSuccess)  // resident channels' instances import their Gram factors
      ps = solve_varlen_fac(slot->plan, n, static_cast<const precode_inst_t*>(slot->d_tbl), base,
                            reinterpret_cast<const float*>(base), s->d_step, s->d_lam, base,
                            slot->d_obj, slot->d_resid, slot->d_flags,
                            n_fac ? reinterpret_cast<float2*>(base) : nullptr,
                            n_fac ? slot->d_fidx : nullptr, st, bucket_n.data());
    for (auto& j : batch) {
      if (e != cudaSuccess || ps != PRECODE_OK) break;
      e = cudaMemcpyAsync(j->d.W_out, base + j->w_off, j->w_bytes, cudaMemcpyDeviceToHost, st);
    }
    if (e == cudaSuccess && ps == PRECODE_OK)
      e = cudaMemcpyAsync(slot->h_obj, slot->d_obj, 4 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ps == PRECODE_OK)
      e = cudaMemcpyAsync(slot->h_resid, slot->d_resid, 4 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && ps == PRECODE_OK)
      e = cudaMemcpyAsync(slot->h_flags, slot->d_flags, 4 * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(slot->done, st);
    lk.lock();
    if (e != cudaSuccess || ps != PRECODE_OK) {
      if (s->error.empty())
        s->error = e != cudaSuccess ? cudaGetErrorString(e) : precode_last_error();
      for (auto& j : batch) j->status = (e != cudaSuccess) ? PRECODE_ECUDA : ps;
    }
    ++s->launches;
    s->factor_instances += n_fac;
    slot->go = true;
    slot->cv.notify_one();
  }
}

// Completion: waits for the slot's launch, stamps its jobs and frees memory.
void slot_loop(precode_server_t s, Slot* slot) {
  DeviceGuard g(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    slot->cv.wait(lk, [&] { return slot->go || s->stop; });
    if (!slot->go && s->stop) return;
    slot->go = false;
    lk.unlock();
    const cudaError_t e = cudaEventSynchronize(slot->done);
    if (e == cudaSuccess)  // per-instance outputs from the pinned staging to the callers
      for (auto& j : slot->jobs) {
        if (j->status != PRECODE_PENDING) continue;
        if (j->d.obj_out) std::memcpy(j->d.obj_out, slot->h_obj + j->first, 4 * j->n);
        if (j->d.resid_out) std::memcpy(j->d.resid_out, slot->h_resid + j->first, 4 * j->n);
        if (j->d.flags_out) std::memcpy(j->d.flags_out, slot->h_flags + j->first, 4 * j->n);
      }
    const double t = now_us();
    lk.lock();
    for (auto& j : slot->jobs) {
      if (j->status == PRECODE_PENDING) j->status = (e == cudaSuccess) ? PRECODE_OK : PRECODE_ECUDA;
      j->done_us = t;
      if (!j->resident) s->arena.release(j->h_off, j->h_bytes);
      s->arena.release(j->w_off, j->w_bytes);
      s->arena.release(j->t_off, j->t_bytes);
      ++s->completed;
      s->instances_done += j->n;
      s->latencies.push_back(j->done_us - j->submit_us);
      s->last_done_us = t;
    }
    slot->jobs.clear();
    slot->busy = false;
    s->cv_dispatch.notify_one();
    s->cv_done.notify_all();
  }
}

double percentile(std::vector<double> v, double q) {
  if (v.empty()) return 0.0;
  std::sort(v.begin(), v.end());
  const double pos = q * (v.size() - 1);
  const size_t i = (size_t)pos;
  const double f = pos - i;
  return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
}

void server_free(precode_server_t s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_dispatch.notify_all();
  for (auto& sl : s->slots) sl->cv.notify_all();
  if (s->dispatcher.joinable()) s->dispatcher.join();
  for (auto& sl : s->slots)
    if (sl->waiter.joinable()) sl->waiter.join();
  DeviceGuard g(s->device);
  for (auto& sl : s->slots) {
    if (sl->stream) cudaStreamSynchronize(sl->stream);
    if (sl->plan) precode_plan_destroy(sl->plan);
    if (sl->stream) cudaStreamDestroy(sl->stream);
    if (sl->done) cudaEventDestroy(sl->done);
    cudaFreeHost(sl->h_tbl);
    cudaFreeHost(sl->h_fidx);
    cudaFree(sl->d_fidx);
    cudaFreeHost(sl->h_obj);
    cudaFreeHost(sl->h_resid);
    cudaFreeHost(sl->h_flags);
    cudaFree(sl->d_tbl);
    cudaFree(sl->d_obj);
    cudaFree(sl->d_resid);
    cudaFree(sl->d_flags);
  }
  cudaFree(s->arena_base);
  cudaFree(s->d_step);
  cudaFree(s->d_lam);
  delete s;
}

}  // namespace
}  // namespace precode

extern "C" {

precode_status_t precode_serve_create(const precode_serve_desc_t* d, precode_server_t* out) {
  if (!d || !out) return fail(PRECODE_EINVAL, "precode_serve_create: NULL argument");
  *out = nullptr;
  if (d->T < 1 || d->T > PRECODE_MAX_T || !d->step || d->n_shapes < 1 || !d->shapes ||
      (d->mode == PRECODE_LAYER_PGD && !d->lam))
    return fail(PRECODE_EINVAL, "precode_serve_create: bad descriptor");
  std::unique_ptr<precode_server_s, void (*)(precode_server_t)> s(new precode_server_s,
                                                                   server_free);
  s->desc = *d;
  s->shapes.assign(d->shapes, d->shapes + d->n_shapes);
  s->desc.shapes = s->shapes.data();
  if (s->desc.n_slots < 1) s->desc.n_slots = 4;
  if (s->desc.max_batch_instances < 1) s->desc.max_batch_instances = 16384;
  s->device = d->device;
  DeviceGuard g(s->device);
  size_t freeb = 0, totalb = 0;
  cudaError_t e = cudaMemGetInfo(&freeb, &totalb);
  if (e != cudaSuccess) return cuda_fail(e, "precode_serve_create: memory query");
  size_t budget = d->device_mem_budget > 0 ? (size_t)d->device_mem_budget : freeb / 2;
  if (budget > freeb) return fail(PRECODE_ENOMEM, "precode_serve_create: budget above free memory");
  if (dev_alloc(&s->arena_base, budget) != cudaSuccess)
    return fail(PRECODE_ENOMEM, "precode_serve_create: arena");
  s->arena.init(budget);
  if (dev_alloc(&s->d_step, 4 * d->T) != cudaSuccess ||
      dev_alloc(&s->d_lam, 4 * d->T) != cudaSuccess)
    return fail(PRECODE_ENOMEM, "precode_serve_create: parameters");
  cudaMemcpy(s->d_step, d->step, 4 * d->T, cudaMemcpyHostToDevice);
  cudaMemcpy(s->d_lam, d->lam ? d->lam : d->step, 4 * d->T, cudaMemcpyHostToDevice);
  precode_desc_t pd{};
  pd.mode = d->mode;
  pd.T = d->T;
  pd.n_shapes = d->n_shapes;
  pd.shapes = s->shapes.data();
  pd.max_instances = s->desc.max_batch_instances;
  pd.cond_threshold = d->cond_threshold;
  pd.flags = d->flags & (PRECODE_PLAN_STEP_NORMALISED | PRECODE_PLAN_GRAPHS | PRECODE_PLAN_AUTOTUNE |
                         PRECODE_PLAN_TENSOR_CORES);
  pd.device = d->device;
  const int64_t cap = s->desc.max_batch_instances;
  for (int i = 0; i < s->desc.n_slots; ++i) {
    // owned by the server from here on, so that a failure below frees what the slot holds
    s->slots.push_back(std::make_unique<Slot>());
    Slot* sl = s->slots.back().get();
    precode_status_t st = precode_plan(&pd, &sl->plan);
    if (st != PRECODE_OK) return st;
    if (cudaStreamCreateWithFlags(&sl->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&sl->done, cudaEventDisableTiming) != cudaSuccess)
      return fail(PRECODE_ECUDA, "precode_serve_create: stream / event");
    // the plan's bucket workspace now, not at the first launch (allocation stalls)
    st = ensure_workspace(sl->plan);
    if (st != PRECODE_OK) return st;
    if (pinned_alloc(&sl->h_tbl, sizeof(precode_inst_t) * cap) != cudaSuccess ||
        pinned_alloc(&sl->h_fidx, sizeof(int64_t) * cap) != cudaSuccess ||
        dev_alloc(&sl->d_fidx, sizeof(int64_t) * cap) != cudaSuccess ||
        pinned_alloc(&sl->h_obj, 4 * cap) != cudaSuccess ||
        pinned_alloc(&sl->h_resid, 4 * cap) != cudaSuccess ||
        pinned_alloc(&sl->h_flags, 4 * cap) != cudaSuccess ||
        dev_alloc(&sl->d_tbl, sizeof(precode_inst_t) * cap) != cudaSuccess ||
        dev_alloc(&sl->d_obj, 4 * cap) != cudaSuccess ||
        dev_alloc(&sl->d_resid, 4 * cap) != cudaSuccess ||
        dev_alloc(&sl->d_flags, 4 * cap) != cudaSuccess)
      return fail(PRECODE_ENOMEM, "precode_serve_create: slot buffers");
  }
  precode_server_t raw = s.get();
  for (auto& sl : s->slots) sl->waiter = std::thread(slot_loop, raw, sl.get());
  s->dispatcher = std::thread(dispatch_loop, raw);
  *out = s.release();
  return PRECODE_OK;
}

precode_status_t precode_serve_channel_create(precode_server_t s, int32_t M, int32_t K,
                                              int32_t n_sc, const void* H, uint64_t* handle) {
  if (!s || !H || !handle || n_sc < 1 || !shape_ok(s->desc.mode, M, K))
    return fail(PRECODE_EINVAL, "precode_serve_channel_create: bad argument");
  const size_t bytes = (size_t)n_sc * K * M * 8;
  size_t off = 0;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->arena.alloc(bytes, &off))
      return fail(PRECODE_ENOMEM, "precode_serve_channel_create: arena full");
  }
  DeviceGuard g(s->device);
  char* const base = static_cast<char*>(s->arena_base);
  cudaError_t e = cudaMemcpy(base + off, H, bytes, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->arena.release(off, bytes);
    return cuda_fail(e, "precode_serve_channel_create: copy");
  }
  Channel ch{M, K, n_sc, off, bytes};
  // The Gram factors of every subcarrier, kept beside H, when the kernel that
  // serves (M, K) imports them: computed here by that kernel, once, so that the
  // jobs on the channel skip the Gram matrix and its inversion.  Without memory
  // for them (or scratch) the channel is kept without factors.
  const Variant* v = s->slots[0]->plan->variant_for(M, K);
  if (v && v->fac && s->desc.mode == PRECODE_LAYER_PROJ) {
    const size_t fac_bytes = (size_t)n_sc * fac_stride(v->KB) * sizeof(float2);
    size_t fac_off = 0, w_off = 0, t_off = 0;
    bool have = false;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->arena.alloc(fac_bytes, &fac_off)) {
        if (s->arena.alloc(bytes, &w_off)) {
          if (s->arena.alloc(4 * (size_t)K, &t_off)) {
            have = true;
          } else {
            s->arena.release(w_off, bytes);
            s->arena.release(fac_off, fac_bytes);
          }
        } else {
          s->arena.release(fac_off, fac_bytes);
        }
      }
    }
    if (have) {
      std::vector<float> ones(K, 1.f);
      cudaStream_t st = nullptr;
      int stride = 0;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + t_off, ones.data(), 4 * (size_t)K, cudaMemcpyHostToDevice, st);
      precode_status_t ps = PRECODE_OK;
      if (e == cudaSuccess)
        ps = plan_export_factors(s->slots[0]->plan, M, K, n_sc, base + off,
                                 reinterpret_cast<float2*>(base + fac_off), base + w_off,
                                 reinterpret_cast<const float*>(base + t_off), st, &stride);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (st) cudaStreamDestroy(st);
      std::lock_guard<std::mutex> lk(s->mu);
      s->arena.release(w_off, bytes);
      s->arena.release(t_off, 4 * (size_t)K);
      if (e != cudaSuccess || ps != PRECODE_OK || stride == 0) {
        s->arena.release(fac_off, fac_bytes);
        if (e != cudaSuccess || ps != PRECODE_OK) {
          s->arena.release(off, bytes);
          return e != cudaSuccess ? cuda_fail(e, "precode_serve_channel_create: factors")
                                  : fail(ps, "precode_serve_channel_create: factors");
        }
      } else {
        ch.fac_off = fac_off;
        ch.fac_bytes = fac_bytes;
        ch.fac_stride = stride;
      }
    }
  }
  std::lock_guard<std::mutex> lk(s->mu);
  *handle = s->next_channel++;
  s->channels[*handle] = ch;
  return PRECODE_OK;
}

precode_status_t precode_serve_channel_destroy(precode_server_t s, uint64_t handle) {
  if (!s) return fail(PRECODE_EINVAL, "precode_serve_channel_destroy: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->channels.find(handle);
  if (it == s->channels.end()) return fail(PRECODE_ENOTFOUND, "precode_serve_channel_destroy");
  // wait until no queued or running job uses it
  s->cv_done.wait(lk, [&] {
    for (auto& kv : s->jobs)
      if (kv.second->d.channel == handle && kv.second->done_us == 0) return false;
    return true;
  });
  s->arena.release(it->second.off, it->second.bytes);
  if (it->second.fac_stride) s->arena.release(it->second.fac_off, it->second.fac_bytes);
  s->channels.erase(it);
  return PRECODE_OK;
}

precode_status_t precode_serve_submit(precode_server_t s, const precode_job_t* job,
                                      uint64_t* ticket) {
  if (!s || !job || !ticket) return fail(PRECODE_EINVAL, "precode_serve_submit: NULL argument");
  const precode_job_t& d = *job;
  if (d.n_sc < 1 || !shape_ok(s->desc.mode, d.M, d.K) || !d.t || !d.W_out ||
      (!d.H && !d.channel))
    return fail(PRECODE_EINVAL, "precode_serve_submit: bad job");
  auto j = std::make_shared<Job>();
  j->d = d;
  j->n = d.n_sc;
  j->w_bytes = (size_t)d.n_sc * d.K * d.M * 8;
  j->h_bytes = j->w_bytes;
  j->t_bytes = 4 * job_t_floats(d);
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->error.empty()) return fail(PRECODE_ECUDA, "precode_serve_submit: server failed: " + s->error);
  if (d.channel) {
    auto it = s->channels.find(d.channel);
    if (it == s->channels.end()) return fail(PRECODE_ENOTFOUND, "precode_serve_submit: channel");
    if (it->second.M != d.M || it->second.K != d.K || it->second.n_sc != d.n_sc)
      return fail(PRECODE_EINVAL, "precode_serve_submit: job shape differs from its channel");
    j->resident = true;
    j->res_h_off = it->second.off;
    j->fac_off = it->second.fac_off;
    j->fac_stride = it->second.fac_stride;
    j->h_bytes = 0;
  }
  const size_t need = ((j->h_bytes + 255) & ~size_t(255)) + ((j->w_bytes + 255) & ~size_t(255)) +
                      ((j->t_bytes + 255) & ~size_t(255));
  if (need > s->arena.size() || j->n > s->desc.max_batch_instances) {
    ++s->rejected;
    return fail(PRECODE_EBUSY, "precode_serve_submit: job larger than the server's memory or slot");
  }
  j->ticket = s->next_ticket++;
  j->submit_us = now_us();
  if (s->submitted == 0) s->first_submit_us = j->submit_us;
  ++s->submitted;
  s->jobs[j->ticket] = j;
  s->queue.push_back(j);
  *ticket = j->ticket;
  s->cv_dispatch.notify_one();
  return PRECODE_OK;
}

static void fill_result(const Job& j, precode_result_t* r) {
  r->status = j.status;
  r->submit_us = j.submit_us;
  r->start_us = j.start_us;
  r->done_us = j.done_us;
  r->latency_us = j.done_us - j.submit_us;
}

precode_status_t precode_serve_poll(precode_server_t s, uint64_t ticket, precode_result_t* r) {
  if (!s || !r) return fail(PRECODE_EINVAL, "precode_serve_poll: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return fail(PRECODE_ENOTFOUND, "precode_serve_poll: unknown ticket");
  if (it->second->done_us == 0) return PRECODE_PENDING;
  fill_result(*it->second, r);
  s->jobs.erase(it);
  return PRECODE_OK;
}

precode_status_t precode_serve_wait(precode_server_t s, uint64_t ticket, int64_t timeout_us,
                                    precode_result_t* r) {
  if (!s || !r) return fail(PRECODE_EINVAL, "precode_serve_wait: NULL argument");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return fail(PRECODE_ENOTFOUND, "precode_serve_wait: unknown ticket");
  auto job = it->second;
  auto pred = [&] { return job->done_us != 0; };
  if (timeout_us < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), pred))
    return fail(PRECODE_ETIMEDOUT, "precode_serve_wait: timed out");
  fill_result(*job, r);
  s->jobs.erase(ticket);
  return PRECODE_OK;
}

precode_status_t precode_serve_stats(precode_server_t s, precode_serve_stats_t* st) {
  if (!s || !st) return fail(PRECODE_EINVAL, "precode_serve_stats: NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = s->submitted;
  st->completed = s->completed;
  st->rejected = s->rejected;
  st->launches = s->launches;
  st->p50_us = percentile(s->latencies, 0.50);
  st->p99_us = percentile(s->latencies, 0.99);
  st->max_us = s->latencies.empty() ? 0.0 : *std::max_element(s->latencies.begin(), s->latencies.end());
  double sum = 0;
  for (double x : s->latencies) sum += x;
  st->mean_us = s->latencies.empty() ? 0.0 : sum / s->latencies.size();
  const double span = s->last_done_us - s->first_submit_us;
  st->precoders_per_s = span > 0 ? s->instances_done / (span * 1e-6) : 0.0;
  st->instances_done = s->instances_done;
  st->factor_instances = s->factor_instances;
  st->bytes_in_use = (int64_t)s->arena.used();
  st->bytes_budget = (int64_t)s->arena.size();
  int busy = 0;
  for (auto& sl : s->slots) busy += sl->busy ? 1 : 0;
  st->slots_busy = busy;
  st->queued = (int32_t)s->queue.size();
  return PRECODE_OK;
}

precode_status_t precode_serve_reset_stats(precode_server_t s) {
  if (!s) return fail(PRECODE_EINVAL, "precode_serve_reset_stats: NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  s->latencies.clear();
  s->submitted = s->completed = s->rejected = s->launches = 0;
  s->instances_done = 0;
  s->first_submit_us = s->last_done_us = 0;
  return PRECODE_OK;
}

precode_status_t precode_serve_destroy(precode_server_t s) {
  if (!s) return fail(PRECODE_EINVAL, "precode_serve_destroy: NULL server");
  {
    std::unique_lock<std::mutex> lk(s->mu);
    // let queued and running work finish
    s->cv_done.wait(lk, [&] {
      if (!s->queue.empty()) return false;
      for (auto& sl : s->slots)
        if (sl->busy) return false;
      return true;
    });
  }
  server_free(s);
  return PRECODE_OK;
}

}  // extern "C"
