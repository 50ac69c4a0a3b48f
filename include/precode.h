/*
 * precode.h -- C ABI of the GB300 deep-unfolded PA-consumption precoder.
 *
 * Method: Feys, Mestre, Peschiera, Rottenberg, "Deep Unfolding for Fast Linear
 * Massive MIMO Precoders under a PA Consumption Model" (VTC2023-Spring,
 * arXiv 2304.12745).
 *
 * Problem (Sec. III, Eq. optim1): for a channel H in C^{K x M} (K users, M
 * antennas) and user targets t_k = sigma_nu sqrt(gamma_k) > 0, find the linear
 * precoder W in C^{K x M} that minimises the PA consumed power
 *     alpha ||W||_{2,1} = alpha sum_m sqrt(sum_k |w_{k,m}|^2)        (Eq. effmodel)
 * subject to H W^T = diag(t).  The library runs T unfolded layers per instance:
 *
 *   PRECODE_LAYER_PGD  (Sec. V, Eq. unfoldednet) -- the paper's layer
 *       V = W - eta_l (W H^T - S) H^*;  W <- prox_{lam_l eta_l ||.||_{2,1}}(V),
 *       prox per antenna column: w_m <- max(0, 1 - tau/||v_m||) v_m (Sec. IV),
 *       W^(0) = H^* (Sec. VI-C).  Constraint enforced only through the penalty.
 *   PRECODE_LAYER_PROJ -- projected layer on the same problem
 *       X = prox_{mu_l ||.||_{2,1}}(W);  W <- P_A(X) = X - (X H^T - S) G^{-T} H^*,
 *       G = H H^H (K x K Gram), W^(0) = S G^{-T} H^* (the ZF precoder).
 *       Every output satisfies H W^T = S up to rounding.
 *
 * Data layout (all buffers caller-owned unless stated):
 *   H, W   complex64 interleaved (re, im) float pairs, instance-major
 *          [B][K][M], row k = user k, column m = antenna m; base 16-byte aligned.
 *   t      float [B][K] (t_stride = K) or one shared [K] vector (t_stride = 0).
 *   step   float [T] device: eta_l (PGD) or mu_l (PROJ).  lam: float [T] device
 *          (PGD only; NULL for PROJ).
 *   obj    float [B] = ||W_T||_{2,1}; resid float [B] = ||H W_T^T - S||_F;
 *   flags  int32 [B] per-instance PRECODE_F_* bits.  obj/resid/flags may be NULL.
 *
 * Conventions: every call is asynchronous on the given stream (cudaStream_t,
 * NULL = legacy default stream); argument errors return PRECODE_EINVAL before
 * any launch; numerical trouble is reported per instance in flags, never as a
 * call failure; no C++ exception crosses this interface; the last error
 * message of the calling thread is available from precode_last_error().
 * A plan may be used from one host thread / stream at a time.
 */
#ifndef PRECODE_H_
#define PRECODE_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* precode_stream_t; /* same type as cudaStream_t */

typedef enum {
  PRECODE_OK = 0,
  PRECODE_EINVAL = 1,    /* bad argument, shape, alignment or size; nothing launched */
  PRECODE_ENOMEM = 2,    /* device or pinned host allocation failed */
  PRECODE_ECUDA = 3,     /* CUDA runtime error (message in precode_last_error) */
  PRECODE_ETIMEDOUT = 4, /* a bounded wait ran out (host wait, or device copy wait) */
  PRECODE_EBUSY = 5,     /* object in use (serving: no slot / memory for the job) */
  PRECODE_PENDING = 6,   /* serving: job not finished yet */
  PRECODE_ENOTFOUND = 7  /* serving: unknown ticket or channel handle */
} precode_status_t;

typedef enum {
  PRECODE_LAYER_PGD = 0,  /* paper layer, Eq. (unfoldednet) */
  PRECODE_LAYER_PROJ = 1  /* shrink + projection onto {H W^T = S} */
} precode_layer_t;

/* per-instance flag bits (int32 flags[b]) */
#define PRECODE_F_FP64_CHOL 1   /* PROJ: equilibrated Gram condition estimate above the
                                   threshold (or FP32 pivot failed): the Gram matrix was
                                   factorised in FP64 (G = L D L^H) and the layers ran in
                                   the orthonormal basis U = D^{-1/2} L^{-1} H of the
                                   channel's row space, targets S~ = D^{-1/2} L^{-1} S
                                   (the same projection, free of G^{-1}'s rounding) */
#define PRECODE_F_SINGULAR 2    /* PROJ: Gram not positive definite even in FP64
                                   (rank(H) < K): W set to 0, obj 0, resid ||S||_F.
                                   The split-FP16 build (K = 8, M = 64) also sets it when
                                   an entry of Q = G^{-T} H^* in its scaled units exceeds
                                   2^13 (an equilibrated Gram condition far beyond FP32
                                   accuracy, met only on the FP64 path) */
#define PRECODE_F_NONFINITE 4   /* NaN/Inf met in the input or the output objective */
#define PRECODE_F_TIMEOUT 8     /* the device-side wait for this instance's channel copy
                                   ran out (about 1 s, or the limit set by
                                   precode_plan_set_debug); W not written */
#define PRECODE_F_INVALID 16    /* uneven batch: descriptor rejected (shape outside every
                                   plan bucket, odd M, K > M for PROJ, negative or odd
                                   offset); W not written */

/* plan flags (precode_desc_t.flags) */
#define PRECODE_PLAN_AUTOTUNE 1u        /* time the kernel variants of each shape at plan
                                           time and keep the fastest (cached in tune_cache) */
#define PRECODE_PLAN_STEP_NORMALISED 2u /* PGD only: use eta_l / L_b with the per-instance
                                           Gershgorin bound L_b = max_k sum_j |G_kj| >=
                                           lambda_max(H H^H) instead of eta_l */
#define PRECODE_PLAN_GRAPHS 4u          /* uneven batches run as one CUDA graph (bucketing
                                           kernel + one solve node per bucket), built on the
                                           first precode_solve_varlen call and re-armed with
                                           new arguments on later calls */

#define PRECODE_PLAN_TENSOR_CORES 8u    /* for shapes with a tensor-core build (8x64, 16x128, 32x256) use it:
                                           contractions as warp MMAs on TF32 operands split
                                           in three terms (products accurate to ~2^-21 rel.);
                                           split-FP16 builds are the defaults for both
                                           layers at K = 8, M = 64 and for the projected
                                           layer with 9..32 users at 64, 128 or 256 antennas
                                           (two FP16 terms per value, ~2^-22 rel., each
                                           instance in exact power-of-two units that keep
                                           it inside the FP16 range) */

#define PRECODE_MAX_K 32
#define PRECODE_MAX_M 256
#define PRECODE_MAX_T 65536

typedef struct {
  int32_t M, K;
} precode_shape_t;

typedef struct {
  int32_t mode;                  /* precode_layer_t */
  int32_t T;                     /* layers, 1..PRECODE_MAX_T */
  int32_t n_shapes;              /* shapes the plan prepares (buckets); >= 1 */
  const precode_shape_t* shapes; /* host array [n_shapes]; 1 <= K <= 32, K <= M <= 256, M even */
  int64_t max_instances;         /* largest B any call will pass (sizes plan workspace) */
  double cond_threshold;         /* PROJ: FP64 path when max(d)/min(d) of the
                                    equilibrated Cholesky pivots exceeds it; <= 0 -> 16.
                                    The FP32 setup's error grows like a few x 2^-24 x
                                    that estimate (about 1e-5 relative at 16 on the
                                    largest bucket); the FP64 path's does not grow */
  uint32_t flags;                /* PRECODE_PLAN_* */
  int32_t device;                /* CUDA device ordinal the plan lives on */
  const char* tune_cache;        /* autotune cache file (read/written), NULL = none */
} precode_desc_t;

typedef struct precode_plan_s* precode_plan_t;

/* One instance of an uneven batch.  Offsets are in elements from the H / W base
 * (complex64 elements, must be even: 16-byte aligned) and from the t base
 * (floats).  Instance b's H is K*M contiguous complex64 values [K][M]. */
typedef struct {
  int64_t h_off;
  int64_t w_off;
  int64_t t_off;
  int32_t M;
  int32_t K;
} precode_inst_t;

/* Create a plan: validates the descriptor, picks a kernel variant per shape
 * (autotuned when PRECODE_PLAN_AUTOTUNE is set, which launches kernels on the
 * device and synchronises), allocates its workspace.  Returns EINVAL on a bad
 * descriptor, ENOMEM / ECUDA on allocation or launch failure. */
precode_status_t precode_plan(const precode_desc_t* desc, precode_plan_t* out);
precode_status_t precode_plan_destroy(precode_plan_t plan);

/* Uniform batch: B instances of one (M, K) (must be one of the plan's shapes or
 * fit one: K <= K_bucket, M <= M_bucket).  All pointers are DEVICE pointers.
 * Runs setup (PROJ: Gram, equilibrated Cholesky, G^{-1}, ZF start) and the T
 * layers of each instance in one persistent kernel, then writes W, obj, resid,
 * flags.  B = 0 is a no-op.  EINVAL: B > max_instances, unaligned pointer,
 * lam == NULL in PGD mode, shape not covered by the plan. */
precode_status_t precode_solve(precode_plan_t plan, int32_t M, int32_t K, int64_t B,
                               const void* H, const float* t, int64_t t_stride,
                               const float* step, const float* lam, void* W, float* obj,
                               float* resid, int32_t* flags, precode_stream_t stream);

/* Same computation from HOST buffers (pinned memory recommended).  When every
 * buffer is page-locked host memory mapped into the device's address space and the
 * shape runs on the projected layer's split-FP16 K = 8, M = 64 build, one kernel reads H and writes W
 * and the outputs in the host buffers directly (zero-copy over the host link).
 * Otherwise the batch is split in chunks whose host->device copy, solve and
 * device->host copy are pipelined over the plan's internal streams.  Both give the
 * device solve's results bit for bit.  step/lam are HOST arrays [T].  Returns after
 * the results are in the host buffers (synchronous). */
precode_status_t precode_solve_host(precode_plan_t plan, int32_t M, int32_t K, int64_t B,
                                    const void* H, const float* t, int64_t t_stride,
                                    const float* step, const float* lam, void* W, float* obj,
                                    float* resid, int32_t* flags);

/* Uneven batch of B instances described by the DEVICE table tbl[B] (any mix of
 * shapes).  A bucketing kernel sorts the instances into the plan's buckets (each
 * plan shape, plus one generic bucket per bucket size that serves any K <= KB,
 * M <= MB), then one persistent solve launch per bucket processes its list; with
 * PRECODE_PLAN_GRAPHS the whole sequence is one CUDA graph launch.  Every
 * instance's result is the same as from precode_solve with its shape.  Outputs
 * obj / resid / flags are indexed by b.  Instances no bucket serves get
 * PRECODE_F_INVALID.  Uses the plan's instance-list workspace (B <= max_instances). */
precode_status_t precode_solve_varlen(precode_plan_t plan, int64_t B, const precode_inst_t* tbl,
                                      const void* H, const float* t, const float* step,
                                      const float* lam, void* W, float* obj, float* resid,
                                      int32_t* flags, precode_stream_t stream);

/* Forward + adjoint through the T layers of a uniform batch (Sec. V: the
 * per-layer parameters are learned by backpropagating the unsupervised cost).
 * Loss = mean_b ( a ||W_T||_{2,1} + ||H W_T^T - S||_F^2 ); writes the DEVICE
 * scalars loss[1], dstep[T] = dLoss/dstep (eta for PGD, mu for PROJ) and, for
 * PGD, dlam[T] = dLoss/dlam.  Parameters at or below zero (clamped to 0 in the
 * layers) get gradient 0.  The forward keeps W every ceil(sqrt(T)) layers in
 * plan workspace (allocated on first use, max_instances sized) and the reverse
 * pass recomputes the layer inputs from them; per-instance partial gradients are
 * averaged in FP64 in a fixed order (bitwise reproducible).  flags [B] optional.
 * With PRECODE_PLAN_TENSOR_CORES at K = 8, M = 64 the forward and adjoint run on
 * the tensor cores: split FP16 for PROJ, split TF32 for PGD (the environment
 * variable PRECODE_TRAIN_TF32, when set, selects split TF32 for PROJ as well).
 * After a first call with the largest B, later calls allocate nothing and make no
 * kernel-attribute or occupancy queries, so they may be captured into a CUDA graph
 * on the given stream.
 * EINVAL: B outside [1, max_instances], NULL loss/dstep, PGD without lam/dlam. */
precode_status_t precode_train_step(precode_plan_t plan, int32_t M, int32_t K, int64_t B,
                                    const void* H, const float* t, int64_t t_stride,
                                    const float* step, const float* lam, float a, float* loss,
                                    float* dstep, float* dlam, int32_t* flags,
                                    precode_stream_t stream);

/* Supervised variant of precode_train_step (Sec. V, supervised cost): the loss
 * is the mean over the batch of the MSE to known ground-truth precoders,
 *     mean_b ||W_T - W_gt||_F^2,
 * and its gradient at the output is 2 (W_T - W_gt); everything else (layers,
 * adjoint, checkpoints, FP64 batch reduction, parameter gradients of zero for
 * parameters at or below zero) is as in precode_train_step.  W_gt: DEVICE
 * complex64 [B][K][M] in W's layout (16-byte aligned), e.g. long-run solutions of
 * Eq. (optim1) computed offline.  An instance whose Gram matrix is singular has
 * W_T = 0 and contributes ||W_gt||_F^2.  EINVAL: NULL W_gt, plus the conditions
 * of precode_train_step. */
precode_status_t precode_train_step_supervised(precode_plan_t plan, int32_t M, int32_t K,
                                               int64_t B, const void* H, const float* t,
                                               int64_t t_stride, const void* W_gt,
                                               const float* step, const float* lam, float* loss,
                                               float* dstep, float* dlam, int32_t* flags,
                                               precode_stream_t stream);

/* Uneven-batch solve that allocates no device memory (the paper has no
 * counterpart: this is a deployment variant of precode_solve_varlen).  For
 * callers that may not call cudaMalloc on their processing path, such as a
 * real-time baseband loop that reserves all memory at start-up, or a host
 * application whose memory manager owns the device.  No plan is needed: `desc`
 * gives mode, T, the shapes (buckets), cond_threshold, device and flags
 * (PRECODE_PLAN_STEP_NORMALISED only; AUTOTUNE, GRAPHS or TENSOR_CORES ->
 * EINVAL); its max_instances is ignored.  Arguments and results are those of
 * precode_solve_varlen with a plan made without flags: the default (FP32)
 * kernel variant of each shape, bit for bit.  A copy wait that runs out is
 * reported only in the instance's flags (PRECODE_F_TIMEOUT): there is no plan
 * whose error counter it could add to.
 * Scratch (bucket instance lists, counters, timeout counter) is one fixed
 * array inside the library, about 2 MiB, that every GPU loading the library
 * holds until exit.  Limits: B <= PRECODE_STATIC_MAX_INSTANCES and at most
 * PRECODE_STATIC_MAX_BUCKETS buckets (the shapes plus one generic bucket per
 * bucket size); larger requests return EINVAL.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) and must come
 * before any stream capture.  All calls share the array: calls whose work
 * overlaps on the GPU (other streams, other threads) race and must be
 * serialised by the caller. */
#define PRECODE_STATIC_MAX_INSTANCES 65536
#define PRECODE_STATIC_MAX_BUCKETS 8
precode_status_t precode_solve_varlen_static(const precode_desc_t* desc, int64_t B,
                                             const precode_inst_t* tbl, const void* H,
                                             const float* t, const float* step, const float* lam,
                                             void* W, float* obj, float* resid, int32_t* flags,
                                             precode_stream_t stream);

/* ---------------------------------------------------------------- serving
 * Continuous batching of precoding jobs (a job = n_sc independent subcarrier
 * channels of one (M, K)).  precode_serve_submit queues a job and returns a
 * ticket at once.  A dispatcher thread admits queued jobs in arrival order into
 * free stream slots while their buffers fit in the server's device arena
 * (admission by free device memory); the jobs admitted together run as one
 * bucketed uneven-batch launch on that slot, overlapping on the device with the
 * other slots' launches.  Jobs arriving while launches run are admitted as soon
 * as a slot and memory free up.  A job's results do not depend on which jobs
 * shared its launch.  Resident channels keep H on the device across jobs.
 * Host buffers of a job must stay valid until its result is polled / waited.
 * H, t and W_out are copied directly: pinned host memory lets those copies
 * overlap with other work (a copy into pageable W_out holds the dispatcher until
 * its launch ends).  obj_out, resid_out and flags_out are staged through the
 * server's pinned buffers and may be pageable. */
typedef struct precode_server_s* precode_server_t;

typedef struct {
  int32_t mode;                  /* precode_layer_t */
  int32_t T;
  const float* step;             /* HOST [T], copied at create */
  const float* lam;              /* HOST [T] (PGD) or NULL */
  int32_t n_shapes;              /* buckets the server prepares (any job shape a bucket holds runs) */
  const precode_shape_t* shapes;
  int32_t n_slots;               /* launches in flight (one stream + plan each); <= 0 -> 4 */
  int64_t max_batch_instances;   /* instances per launch (slot capacity); <= 0 -> 16384 */
  int64_t device_mem_budget;     /* bytes of the job arena; <= 0 -> half the free memory */
  int32_t device;
  double cond_threshold;         /* as in precode_desc_t */
  uint32_t flags;                /* PRECODE_PLAN_* for the slot plans */
} precode_serve_desc_t;

typedef struct {
  int32_t M, K, n_sc;
  const void* H;      /* HOST complex64 [n_sc][K][M]; ignored when channel != 0 */
  const float* t;     /* HOST [n_sc][K], or [K] when t_shared */
  int32_t t_shared;
  void* W_out;        /* HOST complex64 [n_sc][K][M] */
  float* obj_out;     /* HOST [n_sc] or NULL */
  float* resid_out;   /* HOST [n_sc] or NULL */
  int32_t* flags_out; /* HOST [n_sc] or NULL */
  uint64_t channel;   /* resident channel (precode_serve_channel_create) or 0 */
} precode_job_t;

typedef struct {
  precode_status_t status;  /* OK, or the error that hit the job's launch */
  double submit_us, start_us, done_us, latency_us;  /* host steady clock, microseconds */
} precode_result_t;

typedef struct {
  uint64_t submitted, completed, rejected, launches;
  double p50_us, p99_us, max_us, mean_us;  /* submit -> results in host memory */
  double precoders_per_s;                  /* completed instances / (last done - first submit) */
  int64_t instances_done;
  int64_t bytes_in_use, bytes_budget;
  int32_t slots_busy, queued;
  int64_t factor_instances; /* instances launched with their channel's resident Gram factors */
} precode_serve_stats_t;

/* Create the server (arena, one plan + stream per slot, dispatcher and
 * completion threads).  EINVAL bad descriptor, ENOMEM arena / buffers. */
precode_status_t precode_serve_create(const precode_serve_desc_t* desc, precode_server_t* out);
/* Queue a job; returns immediately.  EBUSY if the job can never fit the arena
 * or a slot; ENOTFOUND unknown channel; EINVAL bad job. */
precode_status_t precode_serve_submit(precode_server_t s, const precode_job_t* job,
                                      uint64_t* ticket);
/* PENDING while running; OK fills the result and retires the ticket. */
precode_status_t precode_serve_poll(precode_server_t s, uint64_t ticket, precode_result_t* r);
/* Block until done (timeout_us < 0: no limit); ETIMEDOUT if the limit passes. */
precode_status_t precode_serve_wait(precode_server_t s, uint64_t ticket, int64_t timeout_us,
                                    precode_result_t* r);
precode_status_t precode_serve_stats(precode_server_t s, precode_serve_stats_t* st);
precode_status_t precode_serve_reset_stats(precode_server_t s);
/* Copy n_sc channels [n_sc][K][M] (HOST) to the device once; jobs that name the
 * handle skip the host->device copy of H.  Where the kernel that serves (M, K) keeps
 * Gram factors (the projected layer's split-FP16 K = 8 / M = 64, multi-warp
 * split-FP16 and tcgen05 builds), the channel also keeps each subcarrier's
 * G'^{-T} = (D H H^H D)^{-T} (the Gram inverse of P_A above, with the kernel's
 * per-user power-of-two scales D), computed here once by that kernel, and jobs on it
 * skip the Gram matrix and its inversion: results bitwise the same as a copied
 * channel.  Subcarriers whose Gram matrix takes the FP64 path are set up in full by
 * every job.  ENOMEM: no arena room for H (room for H but not for the factors keeps
 * the channel without them). */
precode_status_t precode_serve_channel_create(precode_server_t s, int32_t M, int32_t K,
                                              int32_t n_sc, const void* H, uint64_t* handle);
/* Waits until no unfinished job uses the channel, then frees it. */
precode_status_t precode_serve_channel_destroy(precode_server_t s, uint64_t handle);
/* Finishes queued and running jobs, then frees everything. */
precode_status_t precode_serve_destroy(precode_server_t s);

/* Number of device-side wait timeouts recorded by the plan's kernels since the
 * plan was created (synchronises the plan's device).  0 in normal operation. */
precode_status_t precode_plan_errors(precode_plan_t plan, uint64_t* count);

/* Failure-detection aid (the paper has no counterpart).  wait_limit_ns sets the
 * limit of each device-side wait of the plan's kernels for an instance's channel
 * copy (0 restores the default of about 1 s).  inject_copy_stall != 0 makes the
 * plan's later launches (solve, uneven solve, train step; not the zero-copy host
 * kernel) issue no channel copy at all, so that every such wait runs out: the
 * waiting group or block then reports PRECODE_F_TIMEOUT in the flags of the
 * instance it was about to solve, adds to precode_plan_errors, waits once more
 * (bounded) and ends without writing W; instances it had not reached keep
 * whatever their output buffers held.  Nothing faults or hangs: no copy is in
 * flight.  This lets a caller exercise its timeout handling without a GPU fault;
 * inject 0 restores normal operation.  A CUDA graph the plan captured earlier
 * (PRECODE_PLAN_GRAPHS) is re-armed with these settings at its next launch.
 * The allocation side has its own aid: with PRECODE_INJECT_ENOMEM=N in the
 * environment, the library's N-th device or page-locked allocation counted from
 * the moment the variable took its current value fails (PRECODE_ENOMEM).
 * EINVAL: NULL plan. */
precode_status_t precode_plan_set_debug(precode_plan_t plan, uint64_t wait_limit_ns,
                                        int32_t inject_copy_stall);

/* Writes the kernel the plan runs for (M, K) into buf (NUL-terminated, as the
 * profiler names it, e.g. "solve_kernel<1, 8, 64, ...>").  EINVAL if the plan
 * does not cover the shape. */
precode_status_t precode_plan_describe(precode_plan_t plan, int32_t M, int32_t K, char* buf,
                                       size_t len);

const char* precode_status_str(precode_status_t status);
/* Message of the last failing call on this host thread ("" if none). */
const char* precode_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PRECODE_H_ */
