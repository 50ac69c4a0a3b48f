"""Benchmark: batched deep-unfolded precoding throughput on GB300.

Workload (the headline): 65,536 independent channels H in C^{8x64} (K=8 users,
M=64 antennas), CN(0,1) entries with 8 dB log-normal per-user gains, unit
targets, T=10 projected layers with per-layer steps mu_t drawn once from
U[0.01, 0.1] (seed 2).  One step = one pass of the whole hot path over the
batch: channel load, Gram matrix, its equilibrated inverse, Q = G^{-T} H^* and
the ZF start, 10 layers (shrink, residual, projection), objective, residual, W
write-back.  It is one persistent kernel launch (the split-FP16 tensor-core
kernel for K = 8, M = 64; --tf32 pins the split-TF32 build instead).  Inputs stay resident in HBM (268 MB of H, larger
than the 129 MB L2; W is another 268 MB), so no L2 flush is needed between steps.

Lines printed (rank 0, one JSON line):
  value      precoders/s from CUDA events over the timed steps (device buffers)
  e2e        the same through precode_solve_host with pinned host buffers
             (host->device, solve, device->host inside the timed region)
  roofline   FP32 FMA-pipe roofline of the solve kernel (the path is
             arithmetic-bound: ~86 flop per HBM byte); on the tensor-core
             kernels also the issued MMA work against the dense tensor peaks
             (all split FP16; all split TF32 with --tf32)
  cpu_baseline  the FP64 oracle on this host's cores, bounded sample
  pa_gap     relative PA-consumption (||W||_{2,1}) difference GPU vs oracle on
             that sample, and the mean PCG of the GPU output
  uneven / train / serving / paper_setting   the other workloads (skipped with
             --no-extras): uneven buckets, learning the steps, Poisson serving, and
             the paper's own setting (PGD 5000 iterations vs 20 unfolded layers;
             per-layer PCG of PGD and of the two unfolded layer maps trained here)
  --impl reference runs the FP64 oracle alone (the CPU comparison arm); --bucket MxK
  and --train run one bucket solve or the training line alone (profiling aids).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2304_12745_gb300 import channels as ch  # noqa: E402

METRIC = ("precoders/s at M=64,K=8,T=10 (fraction of FP32 roofline); PA-power gap vs FP64 "
          "oracle; p99 latency")
UNIT = "precoders/s"


def flops_per_instance(K: int, M: int, T: int, mode: int) -> float:
    """Algorithmic flops of one instance (8 flop per complex multiply-add).

    Paper layer: 2 K^2 M CMAC per layer (residual W H^T and update E H^*).
    Projected layer as computed here: 2 K^2 M per layer (residual and E Q) plus
    setup K^2 M / 2 (Hermitian Gram) + K^3 / 6 (factorisation) + K^2 M (Q)."""
    per_layer = 2 * K * K * M
    setup = 0.0 if mode == 0 else K * K * M / 2 + K ** 3 / 6 + K * K * M
    return 8.0 * (T * per_layer + setup)


def train_flops_per_instance(K: int, M: int, T: int) -> float:
    """Algorithmic flops of one projected-layer train step per instance: the forward
    (setup and T layers), the loss residual and its gradient 2 E_T H^* (one K^2 M
    contraction each) and T reverse layers of two contractions each (g' H'^T, then
    times Q').  The recomputation from checkpoints is not counted."""
    return flops_per_instance(K, M, T, 1) + 8.0 * (2 * K * K * M + T * 2 * K * K * M)


def mma_per_instance(T: int) -> int:
    """Warp MMAs (m16n8k8) the tensor-core kernel issues for one projected-layer
    instance: 48 per 8 x 64 complex contraction (2 real-form blocks x 8 tiles x 3
    split-TF32 terms), two per layer, plus the Gram matrix, Q and Q^T in the
    setup and the final residual."""
    return 96 * T + 48 + 96 + 48


def mma_per_instance_f16(T: int) -> tuple:
    """Warp MMAs the split-FP16 kernel issues for one projected-layer instance:
    (m16n8k16 FP16, m16n8k8 TF32).  Each 8 x 64 complex contraction is 24 FP16 MMAs
    (4 antenna-block pairs x Re/Im H x 3 split terms for a residual; 8 tiles x 3 for
    an update): T layers of two, the final residual, the setup's Gram matrix (one
    residual) and Q, Q^T (8 tiles x 2 products x 3 terms).  No TF32 MMAs remain."""
    return 48 * T + 24 + 24 + 48, 0


def tcgen05_flop_per_instance(T: int, resid: bool) -> tuple:
    """tcgen05.mma work the transposed tcgen05 kernel (32 users x 256 antennas)
    issues for one instance: (flop, pipe slots).  Setup: the Gram matrix and Q^T,
    16 M = N = 128 K = 16 products each; a layer: the residual (16) and the update
    (8 at N = 128, 8 at N = 64); the final residual (16) when it is asked for.  An
    N = 64 product holds the tensor pipe as long as an N = 128 one, so it is one
    slot either way."""
    full = 32 + 24 * T + (16 if resid else 0)
    half = 8 * T
    return full * 2 * 128 * 128 * 16 + half * 2 * 128 * 64 * 16, full + half


_PEAK = {"sms": 152, "mhz": 2070.0, "source": "152 SMs (GB300) x 128 FP32 lanes x 2 flop x 2,070 MHz"}


def set_fp32_peak(sms: int, mhz: float, source: str):
    """The FP32 FMA peak every roofline fraction of the run uses: the device's SM
    count (queried) x 128 FP32 lanes x 2 flop x the SM clock (the median sampled
    under load during the timed region, else the maximum clock)."""
    _PEAK.update(sms=int(sms), mhz=float(mhz), source=source)


def fp32_peak_tflops() -> float:
    """SM count x 128 FP32 lanes x 2 flop x SM clock (see set_fp32_peak)."""
    return _PEAK["sms"] * 128 * 2 * _PEAK["mhz"] * 1e6 / 1e12


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]) if parts[3] not in ("[N/A]", "") else 0.0,
                             parts[5], parts[6], parts[7], parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r[2] > 200.0] or rows
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[3:]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median([r[0] for r in load])), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(load)}


def host_link_peak(torch, nbytes: int = 268 << 20, reps: int = 5) -> dict:
    """Copy-engine bandwidth between page-locked host memory and the device, the
    ceiling of the end-to-end leg: host->device alone, device->host alone, and both
    directions at once on two streams (best of `reps`, CUDA events)."""
    src_h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dst_h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    src_d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    dst_d = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def run(h2d: bool, d2h: bool) -> float:
        best = float("inf")
        for _ in range(reps + 1):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            s1.wait_event(e0)
            s2.wait_event(e0)
            if h2d:
                with torch.cuda.stream(s1):
                    dst_d.copy_(src_h, non_blocking=True)
            if d2h:
                with torch.cuda.stream(s2):
                    dst_h.copy_(src_d, non_blocking=True)
            torch.cuda.current_stream().wait_stream(s1)
            torch.cuda.current_stream().wait_stream(s2)
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1) / 1e3)
        return (int(h2d) + int(d2h)) * nbytes / best / 1e9

    out = {"h2d_gbs": run(True, False), "d2h_gbs": run(False, True), "both_gbs": run(True, True),
           "bytes_per_direction": nbytes,
           "how": "torch copies between page-locked host and device buffers, one stream per "
                  "direction, best of %d, CUDA events" % reps}
    del src_h, dst_h, src_d, dst_d
    return out


def ring_link_rates(torch, ring_bytes: int = 4 << 30, chunk: int = 8 << 20, copies: int = 64,
                    windows: int = 5) -> dict:
    """Copy rates between the device and a page-locked buffer the size of the serving
    load's output ring, as that load uses it: 8 MB copies at random 64 KB-aligned
    offsets, `copies` per window, median over `windows` (CUDA events), taken with the
    server idle.  Recorded beside the serving latencies as the state of the host link
    they were measured under: the device->host rate into such a buffer has been seen
    between ~23 and ~181 GB/s on GB300 hosts after sustained serving load, and at ~181 GB/s
    on runs whose p99 was 12-22 ms, so it does not by itself explain the tail."""
    host = torch.empty(ring_bytes, dtype=torch.uint8, pin_memory=True)
    dev = torch.empty(chunk, dtype=torch.uint8, device="cuda")
    rng = np.random.default_rng(3)
    st = torch.cuda.current_stream()

    def window(d2h: bool) -> float:
        offs = rng.integers(0, (ring_bytes - chunk) // 65536, copies) * 65536
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        for o in offs:
            if d2h:
                host[int(o):int(o) + chunk].copy_(dev, non_blocking=True)
            else:
                dev.copy_(host[int(o):int(o) + chunk], non_blocking=True)
        e1.record(st)
        torch.cuda.synchronize()
        return copies * chunk / (e0.elapsed_time(e1) / 1e3) / 1e9

    window(True)
    d2h = [window(True) for _ in range(windows)]
    h2d = [window(False) for _ in range(windows)]
    del host, dev
    return {"d2h_gbs": float(np.median(d2h)), "d2h_gbs_min": float(min(d2h)),
            "h2d_gbs": float(np.median(h2d))}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_baseline(H, t, mu, budget_s: float = 10.0):
    """FP64 oracle throughput on this host's cores over a bounded sample: the
    workload's instances in order (wrapping around) until ~budget_s of wall time."""
    import oracle
    oracle.build()
    nthreads = os.cpu_count() or 1
    # one thread first (the per-core rate), then one thread per core
    n1 = min(len(H), 64)
    t0 = time.perf_counter()
    oracle.batch_forward(1, H[:n1].astype(np.complex128), t[:n1].astype(np.float64),
                         mu.astype(np.float64), nthreads=1)
    single = n1 / max(time.perf_counter() - t0, 1e-9)
    n0 = min(len(H), 8 * nthreads)
    t0 = time.perf_counter()
    oracle.batch_forward(1, H[:n0].astype(np.complex128), t[:n0].astype(np.float64),
                         mu.astype(np.float64), nthreads=nthreads)
    rate0 = n0 / max(time.perf_counter() - t0, 1e-6)
    chunk = int(min(len(H), max(n0, rate0 * budget_s / 4)))
    done, first_obj = 0, None
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        lo = done % len(H)
        hi = min(lo + chunk, len(H))
        W, obj, res, st = oracle.batch_forward(1, H[lo:hi].astype(np.complex128),
                                               t[lo:hi].astype(np.float64), mu.astype(np.float64),
                                               nthreads=nthreads)
        if first_obj is None:
            first_obj = (lo, obj)
        done += hi - lo
    dt = time.perf_counter() - t0
    return {"value": done / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"{done} instances of the workload in order (wrapping), FP64 projected "
                      f"layers, {nthreads} threads over contiguous ranges, {dt:.1f} s",
            "single_thread_value": single}, first_obj


def bench_uneven(torch, capi, Plan, inst_table):
    """Uneven workload: 32,768 instances, (M, K) uniform over the four buckets,
    Rician channels, T = 10, one CUDA-graph launch (bucketing + one solve per bucket).
    Also each bucket alone (a uniform solve of its instances) with its FP32 roofline
    fraction."""
    B, T = 32768, 10
    shapes = ch.uneven_shapes(B, seed=3)
    pool, h_off = ch.uneven_channels(shapes, seed=3)
    t_off = np.concatenate([[0], np.cumsum(shapes[:, 1])[:-1]]).astype(np.int64)
    Hd = torch.from_numpy(pool).cuda()
    td = torch.ones(int(shapes[:, 1].sum()), device="cuda")
    mu = torch.from_numpy(ch.uniform_steps(T, 0.01, 0.1, seed=2)).cuda()
    plan = Plan(capi.LAYER_PROJ, T, [tuple(x) for x in ch.UNEVEN_SHAPES], B, graphs=True,
                autotune=True)
    tbl = inst_table(h_off, h_off, t_off, shapes[:, 0], shapes[:, 1]).cuda()
    W = torch.empty_like(Hd)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    ms = timed(lambda: plan.solve_varlen(tbl, Hd, td, mu, W=W))
    fl = plan.solve_varlen(tbl, Hd, td, mu, W=W)[3]
    fp64 = int(((fl.cpu().numpy() & capi.F_FP64_CHOL) != 0).sum())
    plan.close()
    peak = fp32_peak_tflops()
    per, flops_total = {}, 0.0
    for (M, K) in ch.UNEVEN_SHAPES:
        idx = np.nonzero((shapes[:, 0] == M) & (shapes[:, 1] == K))[0]
        n = len(idx)
        Hb = torch.from_numpy(pool[h_off[idx][:, None] + np.arange(K * M)[None, :]]
                              .reshape(n, K, M)).cuda()
        tb = torch.ones(n, K, device="cuda")
        pb = Plan(capi.LAYER_PROJ, T, [(M, K)], n, autotune=True, tensor_cores=True)
        out = (torch.empty_like(Hb), torch.empty(n, device="cuda"), None,
               torch.empty(n, device="cuda", dtype=torch.int32))
        msb = timed(lambda: pb.solve(Hb, tb, mu, out=out))
        fpi = flops_per_instance(K, M, T, 1)
        flops_total += fpi * n
        kname = capi.precode_plan_describe(pb.handle, M, K)
        per[f"{M}x{K}"] = {"instances": n, "precoders_per_s": n / (msb / 1e3), "ms": msb,
                           "fp32_roofline_frac": fpi * n / (msb / 1e3) / 1e12 / peak,
                           "kernel": kname}
        if kname.startswith("solve_tgt_kernel"):  # its products run on the tensor pipe
            fl, slots = tcgen05_flop_per_instance(T, resid=False)
            bf16 = measured_peaks().get("bf16_tflops", 1900.0)
            issued = fl * n / (msb / 1e3) / 1e12
            per[f"{M}x{K}"]["tensor"] = {
                "issued_tflops": issued, "peak_tflops": bf16, "frac": issued / bf16,
                "flop_per_instance": fl, "mma_slots_per_instance": slots,
                "note": "issued tcgen05.mma work (FP16, split hi / lo) against the measured "
                        "bf16 burst peak (of measured); the FP32 fraction above counts "
                        "the algorithmic complex flops against the FP32 roofline"}
        pb.close()
    return {"workload": "uneven: 32,768 instances, (M,K) uniform over (32,4),(64,8),(128,16),"
                        "(256,32), Rician ULA per instance, T=10, one CUDA graph per call",
            "precoders_per_s": B / (ms / 1e3), "ms_per_call": ms,
            "fp32_roofline_frac": flops_total / (ms / 1e3) / 1e12 / peak,
            "fp64_fallbacks": fp64, "buckets": per}


def bench_train(torch, capi):
    """Differentiation workload: Adam over mu_1..mu_10 for 200 batches of 8,192
    i.i.d. CN(0,1) channels C^{8x64}; loss = mean PA objective + residual penalty."""
    from paper_2304_12745_gb300.training import UnfoldedTrainer
    K, M, T, Bt, steps = 8, 64, 10, 8192, 200
    tr = UnfoldedTrainer(capi.LAYER_PROJ, T, K, M, Bt, a=1.0, lr=1e-3,
                         init_step=list(ch.fixed_workload_steps(T)), graphs=True)
    t = torch.ones(K, device="cuda")
    nb = 8
    batches = [tr.make_batch(i, seed=4) for i in range(nb)]  # 8 resident batches, cycled
    # the first step on each batch runs eagerly and captures that batch's graph
    first = tr.train_step(batches[0], t)
    for i in range(1, nb):
        tr.train_step(batches[i], t)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    last = None
    for i in range(nb, steps):
        last = tr.train_step(batches[i % nb], t, sync=False)  # no host round trip per step
    e1.record()
    torch.cuda.synchronize()
    last = float(last)
    ms = e0.elapsed_time(e1) / (steps - nb)
    mu = tr.step.detach().cpu().numpy()
    tr.plan.close()
    del batches
    # the train-step launch alone (forward + adjoint kernel and batch reductions) on
    # 65,536 resident instances, against the FP32 roofline
    from paper_2304_12745_gb300.precoder import Plan
    Bk = 65536
    Hk = torch.from_numpy(ch.rayleigh(Bk, K, M, seed=1)).cuda()
    tk = torch.ones(Bk, K, device="cuda")
    muk = torch.from_numpy(ch.fixed_workload_steps(T)).cuda()
    pk = Plan(capi.LAYER_PROJ, T, [(M, K)], Bk, tensor_cores=True)
    lk, dk = torch.empty(1, device="cuda"), torch.empty(T, device="cuda")
    stream = torch.cuda.current_stream()

    def kstep():
        capi.precode_train_step(pk.handle, M, K, Bk, Hk, tk, K, muk, None, 1.0, lk, dk, None,
                                None, stream.cuda_stream)

    for _ in range(3):
        kstep()
    torch.cuda.nvtx.range_push("prof")  # the launch a profiler captures
    kstep()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k0.record(stream)
    for _ in range(20):
        kstep()
    k1.record(stream)
    torch.cuda.synchronize()
    kms = k0.elapsed_time(k1) / 20
    pk.close()
    fpi = train_flops_per_instance(K, M, T)
    kernel = {"instances": Bk, "ms_per_launch": kms, "instances_per_s": Bk / (kms / 1e3),
              "flop_per_instance": fpi,
              "fp32_roofline_frac": fpi * Bk / (kms / 1e3) / 1e12 / fp32_peak_tflops(),
              "note": "precode_train_step alone (one train kernel + FP64 batch reductions); "
                      "flops without the checkpoint recomputation"}
    return {"workload": "train: 200 Adam steps x 8,192 instances C^{8x64}, CN(0,1), T=10, lr 1e-3; "
                        "one CUDA graph per resident batch, the last 192 steps timed",
            "instances_per_s": Bt / (ms / 1e3), "ms_per_step": ms, "loss_first": first,
            "loss_last": last, "mu_learned": [float(x) for x in mu], "kernel": kernel}, mu


def sum_rate_per_channel(torch, H, W, sigma: float = 1.0):
    """R_sum = sum_k log2(1 + SINR_k) per channel (Sec. VI-B), SINR_k =
    |[H W^T]_kk|^2 / (sum_{j != k} |[H W^T]_kj|^2 + sigma^2); evaluation of the
    solver's outputs, not part of the solve."""
    E = torch.bmm(H, W.transpose(1, 2))  # [B][K][K], row k: user k's received gains
    p = E.abs() ** 2
    sig = torch.diagonal(p, dim1=1, dim2=2)
    intf = p.sum(dim=2) - sig
    return torch.log2(1 + sig / (intf + sigma * sigma)).sum(dim=1)


def bench_paper_setting(torch, capi, max_epochs: int = 200, patience: int = 5):
    """The paper's own setting and recipe (Sec. VI): K = 8, M = 64, i.i.d. CN(0,1)
    channels, gamma = 10 dB per user (t = sqrt(10), sigma_nu = 1), lambda = 1/15,
    I = 20 layers, W^(0) = H^* for the paper layer.
    speed:   the classical PGD (5,000 iterations, constant eta = 1/L~, lambda = 1/15)
             through the same paper-layer kernel, next to the 20-layer unfolded
             network, 8,192 channels per call;
    quality: Sec. VI-A's training recipe: 10^5 training channels, Adam with batch 64
             and learning rate 1e-3, epochs of 1,562 steps over a fresh permutation,
             at most 200 epochs, early stopping when the loss on 5,000 validation
             channels has not improved for `patience` epochs (the best parameters are
             kept); then per-layer PCG, sum rate and constraint residual on 5,000
             test channels (Sec. VI-B) for PGD, the unfolded paper layer trained
             unsupervised (cost lambda ||W||_{2,1} + ||H W^T - S||_F^2) and supervised
             (MSE to labels), and the unfolded projected layer trained unsupervised.
             Labels: the constrained optimum approximated on the GPU by 4,000
             projected layers with shrink mu_t = 0.1 / sqrt(t) (within ~0.1 % of the
             ADMM optimum's objective), in place of the paper's CVXPY solutions.
             Target: the FP64 oracle's ADMM optimum of the same test channels
             (tests/golden/quality_reference.json), the paper's 1.1160."""
    from paper_2304_12745_gb300.precoder import Plan
    from paper_2304_12745_gb300.training import UnfoldedTrainer
    K, M, T = 8, 64, 20
    amp = math.sqrt(10.0)
    lam_pgd = 1.0 / 15
    eta = ch.paper_eta(K, M)
    dev = "cuda"
    tK = torch.full((K,), amp, device=dev)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # speed: PGD 5,000 iterations vs the 20-layer network (same kernel, same batch)
    Bs = 8192
    Hs = torch.from_numpy(ch.rayleigh(Bs, K, M, seed=40)).cuda()
    speed = {}
    for name, TT in (("pgd_5000", 5000), ("unfolded_20", T)):
        pl = Plan(capi.LAYER_PGD, TT, [(M, K)], Bs, tensor_cores=True)
        st = torch.full((TT,), eta, device=dev)
        lm = torch.full((TT,), lam_pgd, device=dev)
        ms = timed(lambda: pl.solve(Hs, tK, st, lm), 2 if TT > 100 else 20)
        speed[name] = {"ms_per_call": ms, "precoders_per_s": Bs / (ms / 1e3),
                       "kernel": capi.precode_plan_describe(pl.handle, M, K)}
        pl.close()
    speed["ratio"] = speed["pgd_5000"]["ms_per_call"] / speed["unfolded_20"]["ms_per_call"]
    del Hs

    # data (Sec. VI-A) and labels
    Htr = torch.from_numpy(ch.paper_set("train")).cuda()
    Hva = torch.from_numpy(ch.paper_set("validation")).cuda()
    Hte = torch.from_numpy(ch.paper_set("test")).cuda()
    T_long = 4000
    mu_long = (0.1 / torch.sqrt(torch.arange(1, T_long + 1, device=dev, dtype=torch.float32))).contiguous()
    pl_long = Plan(capi.LAYER_PROJ, T_long, [(M, K)], len(Htr), tensor_cores=True)
    t0 = time.perf_counter()
    lab_tr = pl_long.solve(Htr, tK, mu_long, want_resid=False)[0]
    lab_va = pl_long.solve(Hva, tK, mu_long, want_resid=False)[0]
    _, obj_long_te, _, _ = pl_long.solve(Hte, tK, mu_long, want_resid=False)
    torch.cuda.synchronize()
    label_s = time.perf_counter() - t0
    pl_long.close()
    pz = Plan(capi.LAYER_PROJ, 1, [(M, K)], len(Hte), tensor_cores=True)
    _, obj_zf, _, _ = pz.solve(Hte, tK, torch.zeros(1, device=dev))
    pz.close()

    def val_loss(mode, st, lm, kind, plan):
        W, obj, res, _ = plan.solve(Hva, tK, st.detach().contiguous(),
                                    None if lm is None else lm.detach().contiguous())
        if kind == "supervised":
            return float(((W - lab_va).abs() ** 2).sum(dim=(1, 2)).mean())
        return float((lam_pgd * obj + res * res).mean())

    def train(mode, kind):
        bs = 64
        tr = UnfoldedTrainer(mode, T, K, M, bs, a=lam_pgd, lr=1e-3, graphs=True)
        vplan = Plan(mode, T, [(M, K)], len(Hva), tensor_cores=True)
        Hbuf = torch.empty(bs, K, M, dtype=torch.complex64, device=dev)
        Lbuf = torch.empty_like(Hbuf) if kind == "supervised" else None
        gen = torch.Generator().manual_seed(7)
        steps_per_epoch = len(Htr) // bs
        best = (val_loss(mode, tr.step, tr.lam, kind, vplan), tr.step.detach().clone(),
                None if tr.lam is None else tr.lam.detach().clone(), 0)
        history, bad, epoch = [best[0]], 0, 0
        t0 = time.perf_counter()
        for epoch in range(1, max_epochs + 1):
            perm = torch.randperm(len(Htr), generator=gen).to(dev)
            for i in range(steps_per_epoch):
                idx = perm[i * bs:(i + 1) * bs]
                torch.index_select(Htr, 0, idx, out=Hbuf)
                if Lbuf is not None:
                    torch.index_select(lab_tr, 0, idx, out=Lbuf)
                tr.train_step(Hbuf, tK, sync=False, labels=Lbuf)
            vl = val_loss(mode, tr.step, tr.lam, kind, vplan)
            history.append(vl)
            if vl < best[0] * (1 - 1e-6):
                best, bad = (vl, tr.step.detach().clone(),
                             None if tr.lam is None else tr.lam.detach().clone(), epoch), 0
            else:
                bad += 1
                if bad >= patience:
                    break
        torch.cuda.synchronize()
        secs = time.perf_counter() - t0
        vplan.close()
        tr.plan.close()
        return {"mode": mode, "steps": best[1], "lams": best[2], "epochs": epoch,
                "best_epoch": best[3], "adam_steps": epoch * steps_per_epoch, "train_s": secs,
                "val_loss_per_epoch": history}

    runs = {"ufpgd_unsupervised": train(capi.LAYER_PGD, "unsupervised"),
            "ufpgd_supervised": train(capi.LAYER_PGD, "supervised"),
            "ufpgd_projected": train(capi.LAYER_PROJ, "unsupervised")}
    runs["pgd"] = {"mode": capi.LAYER_PGD, "steps": torch.full((T,), eta, device=dev),
                   "lams": torch.full((T,), lam_pgd, device=dev)}

    s_norm = amp * math.sqrt(K)
    methods = {}
    for name, r in runs.items():
        pcg, rsum, res = [], [], []
        for TT in range(1, T + 1):
            pl = Plan(r["mode"], TT, [(M, K)], len(Hte), tensor_cores=True)
            W, obj, rsd, _ = pl.solve(Hte, tK, r["steps"][:TT].contiguous(),
                                      None if r["lams"] is None else r["lams"][:TT].contiguous())
            pcg.append(float((obj_zf / obj).mean()))
            rsum.append(float(sum_rate_per_channel(torch, Hte, W).mean()))
            res.append(float(rsd.mean()) / s_norm)
            pl.close()
        m = {"pcg_per_layer": pcg, "sum_rate_per_layer": rsum, "rel_residual_per_layer": res,
             "steps": [float(x) for x in r["steps"].cpu()],
             "lambdas": None if r["lams"] is None else [float(x) for x in r["lams"].cpu()]}
        for k in ("epochs", "best_epoch", "adam_steps", "train_s", "val_loss_per_epoch"):
            if k in r:
                m[k] = r[k]
        methods[name] = m
    try:
        ref = json.load(open(os.path.join(ROOT, "tests", "golden", "quality_reference.json")))
    except Exception:
        ref = {}
    return {"workload": "paper setting: K=8, M=64, CN(0,1), gamma=10 dB, I=20; PGD 5000 it. vs "
                        "20 unfolded layers; Sec. VI-A training recipe; per-layer metrics on "
                        "5,000 test channels",
            "speed": speed,
            "quality": {
                "recipe": "10^5 training / 5,000 validation / 5,000 test channels (seeded "
                          "CN(0,1)); Adam, batch 64, lr 1e-3, epochs of 1,562 steps, early "
                          f"stopping after {patience} epochs without validation improvement "
                          f"(at most {max_epochs}); lambda = 1/15 in PGD and in the "
                          "unsupervised cost; supervised labels from 4,000 projected layers "
                          "with mu_t = 0.1/sqrt(t) on the GPU",
                "pcg_20": {k: v["pcg_per_layer"][-1] for k, v in methods.items()},
                "sum_rate_20": {k: v["sum_rate_per_layer"][-1] for k, v in methods.items()},
                "target": {"pcg_admm_optimum_test_set": ref.get("pcg_mean"),
                           "sum_rate_admm_optimum_test_set": ref.get("sum_rate_mean"),
                           "source": "tests/golden/quality_reference.json (FP64 oracle ADMM)",
                           "pcg_gpu_long_run_labels": float((obj_zf / obj_long_te).mean()),
                           "label_generation_s": label_s},
                "methods": methods,
                "paper_printed": {"pcg_ufpgd_unsupervised_20": 1.0915, "pcg_cvx_optimum": 1.1160,
                                  "pcg_pgd_20": "about 1", "sum_rate_target": 27.68}}}


def bench_serve(capi, mu, duration_s: float = 2.0, n_runs: int = 3):
    """Serving workload: Poisson arrivals at 2,000 jobs/s, M in {64,128,256},
    K in {4..32}, N_sc in {64,...,1024}, Rician, T = 10 with the learned steps."""
    from paper_2304_12745_gb300.serving import Server, poisson_load
    # buckets: every job shape (M in {64,128,256}, any K <= 32) fits a user-padded
    # tensor-core bucket of 8, 16, 24 or 32 users
    shapes = [(m, k) for m in (64, 128, 256) for k in (8, 16, 24, 32)]
    s = Server(capi.LAYER_PROJ, mu, shapes=shapes, n_slots=6, max_batch_instances=65536,
               device_mem_budget=24 << 30, flags=capi.PLAN_TENSOR_CORES)
    # warm-up: one job per bucket (every kernel the load can use is loaded and its
    # first launch done), then a short Poisson run
    rng = np.random.default_rng(10)
    warm = []
    for m in (64, 128, 256):
        for k in (4, 12, 20, 28, 8, 16, 24, 32):
            H = ch.rician_ula(64, k, m, seed=int(rng.integers(1 << 30)))
            warm.append(s.submit(H, np.ones(k, np.float32)))
    for j in warm:
        j.wait()
    poisson_load(s, 500.0, 0.2, seed=11)
    import torch
    link_before = ring_link_rates(torch)
    runs = []
    for r in range(n_runs):  # independent Poisson runs back to back (seeds 12, 13, ...)
        s.reset_stats()
        st = poisson_load(s, 2000.0, duration_s, seed=12 + r)
        runs.append({"p50_ms": st["p50_us"] / 1e3, "p99_ms": st["p99_us"] / 1e3,
                     "max_ms": st["max_us"] / 1e3, "precoders_per_s": st["precoders_per_s"],
                     "jobs": st["jobs"], "achieved_jobs_per_s": st["achieved_rate_per_s"],
                     "launches": st["launches"]})
    link_after = ring_link_rates(torch)
    s.close()
    med = lambda k: float(np.median([r[k] for r in runs]))  # noqa: E731
    return {"workload": "serve: Poisson 2,000 jobs/s, %d runs of %.1f s; M in {64,128,256}, "
                        "K in {4..32}, N_sc in {64,128,256,512,1024}; Rician; T=10, learned mu"
                        % (n_runs, duration_s),
            "p50_ms": med("p50_ms"), "p99_ms": med("p99_ms"), "max_ms": max(r["max_ms"] for r in runs),
            "p99_ms_per_run": [r["p99_ms"] for r in runs],
            "precoders_per_s": med("precoders_per_s"), "jobs": sum(r["jobs"] for r in runs),
            "achieved_jobs_per_s": med("achieved_jobs_per_s"), "runs": runs,
            "ring_link": {"before_runs": link_before, "after_runs": link_after,
                          "how": "8 MB copies at random offsets of a page-locked 4 GB buffer "
                                 "(the output ring's size), median of 5 windows of 64, with "
                                 "the server idle"},
            "note": "p50 / p99 / precoders per s: median over the runs; max: over all runs"}


def bench_resident(capi, mu, reps: int = 20) -> dict:
    """Jobs on resident channels (H and each subcarrier's Gram factors kept on the
    device) against the same jobs with H copied in: median latency of a job alone on
    the server (submit -> results in host memory), 1,024 subcarriers."""
    from paper_2304_12745_gb300.serving import JobHandle, Server, pinned, touch_by_device
    shapes = [(m, k) for m in (64, 128, 256) for k in (8, 16, 24, 32)]
    s = Server(capi.LAYER_PROJ, mu, shapes=shapes, n_slots=2, max_batch_instances=65536,
               device_mem_budget=8 << 30, flags=capi.PLAN_TENSOR_CORES)
    out = {}
    for M, K in ((64, 8), (256, 32)):
        n = 1024
        H = ch.rician_ula(n, K, M, seed=77 + K)
        cid = s.channel(H)
        # page-locked job buffers, touched by the device once (as poisson_load's)
        Hp = pinned(H.size, np.complex64).reshape(H.shape)
        Hp[:] = H
        Wp = pinned(H.size, np.complex64).reshape(H.shape)
        ones = pinned(K, np.float32)
        ones[:] = 1.0
        touch_by_device(Hp, Wp, ones)
        lat = {"copied": [], "resident": []}
        for r in range(reps + 2):
            for kind in ("copied", "resident"):
                arrays = {"H": Hp, "t": ones, "W": Wp, "obj": np.empty(n, np.float32),
                          "resid": None, "flags": np.empty(n, np.int32)}
                job = capi.Job(M, K, n, capi.ptr(Hp) if kind == "copied" else None, capi.ptr(ones), 1,
                               capi.ptr(Wp), capi.ptr(arrays["obj"]), None, capi.ptr(arrays["flags"]),
                               0 if kind == "copied" else cid)
                res = JobHandle(s, capi.precode_serve_submit(s.handle, job), arrays).wait()
                if r >= 2:
                    lat[kind].append(res.latency_us / 1e3)
        out[f"{M}x{K}x{n}"] = {"copied_ms": float(np.median(lat["copied"])),
                               "resident_ms": float(np.median(lat["resident"])),
                               "h_bytes": int(H.nbytes)}
        s.release_channel(cid)
    st = s.stats()
    s.close()
    out["factor_instances"] = int(st["factor_instances"])
    out["note"] = ("resident: H and its Gram factors stay on the device, so a job skips the "
                   "host->device copy of H and the kernels skip the Gram matrix and its "
                   "inversion; page-locked host buffers; median of %d jobs alone on the "
                   "server" % reps)
    return out


def run_bucket(args):
    """One bucket alone (profiling aid): B Rician channels C^{K x M} (seed 5), T = 10
    projected layers, autotuned plan; two solves, then one inside an NVTX range."""
    import torch
    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan
    M, K = (int(x) for x in args.bucket.lower().split("x"))
    B, T = args.bucket_instances, 10
    H = torch.from_numpy(ch.rician_ula(B, K, M, seed=5)).cuda()
    t = torch.ones(B, K, device="cuda")
    mu = torch.from_numpy(ch.uniform_steps(T, 0.01, 0.1, seed=2)).cuda()
    cache = None
    if args.tf32:  # pin the bucket's split-TF32 tensor-core build
        kw = -(-K // 8)
        minb = {64: {1: 16, 2: 8, 3: 5, 4: 4}, 128: {1: 12, 2: 6, 3: 4, 4: 3},
                256: {1: 8, 2: 4, 3: 2, 4: 2}}[M][kw]
        cache = os.path.join(tempfile.mkdtemp(), "tune.txt")
        with open(cache, "w") as f:
            f.write(f"{torch.cuda.get_device_name(0)}|{capi.LAYER_PROJ}|{K}|{M}\t"
                    f"{8 * kw}x{M}/{kw}x8/jc8/w{kw}/b{minb}/split/tc/exact\n")
    plan = Plan(capi.LAYER_PROJ, T, [(M, K)], B, autotune=True, tune_cache=cache)
    out = (torch.empty_like(H), torch.empty(B, device="cuda"), None,
           torch.empty(B, device="cuda", dtype=torch.int32))
    for _ in range(2):
        plan.solve(H, t, mu, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("prof")
    e0.record()
    plan.solve(H, t, mu, out=out)
    e1.record()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    print(json.dumps({"bucket": f"{M}x{K}", "instances": B, "ms": e0.elapsed_time(e1),
                      "kernel": capi.precode_plan_describe(plan.handle, M, K)}))
    plan.close()


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    oracle.build()
    wl = ch.WORKLOADS["fixed"]
    nthreads = os.cpu_count() or 1
    n = min(wl.B, max(64, 24 * nthreads))
    H = ch.lognormal(n, wl.K, wl.M, seed=wl.seed).astype(np.complex128)
    t = ch.targets(n, wl.K).astype(np.float64)
    mu = ch.fixed_workload_steps(wl.T).astype(np.float64)
    for _ in range(args.warmup):
        oracle.batch_forward(1, H[:nthreads], t[:nthreads], mu, nthreads=nthreads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.batch_forward(1, H, t, mu, nthreads=nthreads)
    dt = time.perf_counter() - t0
    value = n * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": "fixed: 65,536 x C^{8x64}, 8 dB log-normal Rayleigh, T=10 "
                                   "projected layers, mu_t ~ U[0.01,0.1]",
                       "sample_per_step": n, "layer": "projected"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"{n} instances of the workload per step (FP64 oracle, "
                                       f"{nthreads} threads)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the uneven, training and serving sub-benchmarks")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the default kernel variant (no tuning launches; for profiling)")
    ap.add_argument("--tf32", action="store_true",
                    help="pin the headline shape (or the --bucket shape) to its split-TF32 "
                         "tensor-core build (the split-FP16 builds are the defaults); for "
                         "profiling and comparison")
    ap.add_argument("--ffma", action="store_true",
                    help="run the headline on the FP32 FFMA kernel (no tensor cores); for "
                         "profiling and comparison")
    ap.add_argument("--bucket", default=None, metavar="MxK",
                    help="profiling aid: solve one uniform bucket of Rician channels (autotuned "
                         "plan), the last solve inside an NVTX range 'prof', print one line, exit")
    ap.add_argument("--bucket-instances", type=int, default=4096)
    ap.add_argument("--paper", action="store_true",
                    help="run only the paper-setting sub-benchmark (speed of PGD-5000 vs 20 "
                         "unfolded layers, and the Sec. VI-A training recipe with per-layer "
                         "PCG / sum rate on the test set), print its line, exit")
    ap.add_argument("--train", action="store_true",
                    help="run only the training sub-benchmark (the 200 Adam steps, then the "
                         "train-step launch alone with one launch inside an NVTX range 'prof'), "
                         "print its line, exit")
    return ap


def main():
    args = _parser().parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.bucket:
        return run_bucket(args)
    if args.train:
        import torch
        from paper_2304_12745_gb300 import capi
        line, _ = bench_train(torch, capi)
        print(json.dumps(line))
        return
    if args.paper:
        import torch
        from paper_2304_12745_gb300 import capi
        print(json.dumps(bench_paper_setting(torch, capi)))
        return

    import torch
    import torch.distributed as dist

    from paper_2304_12745_gb300 import capi
    from paper_2304_12745_gb300.precoder import Plan

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    wl = ch.WORKLOADS["fixed"]
    B, K, M, T = wl.B, wl.K, wl.M, wl.T
    # weak scaling: each rank solves its own 65,536-instance shard
    H = ch.lognormal(B, K, M, seed=wl.seed + 1000 * rank)
    t = ch.targets(B, K)
    mu = ch.fixed_workload_steps(T)
    if args.tf32:  # an autotune cache entry naming the split-TF32 build
        cache = os.path.join(tempfile.mkdtemp(), "tune.txt")
        with open(cache, "w") as f:
            f.write(f"{torch.cuda.get_device_name(local)}|{capi.LAYER_PROJ}|{K}|{M}\t"
                    f"{K}x{M}/4x8/jc8/w4/b3/split/tc/exact\n")
        plan = Plan(capi.LAYER_PROJ, T, [(M, K)], B, autotune=True, tensor_cores=True,
                    tune_cache=cache)
    else:
        plan = Plan(capi.LAYER_PROJ, T, [(M, K)], B, autotune=not args.no_autotune,
                    tensor_cores=not args.ffma)
    Hd = torch.from_numpy(H).cuda()
    td = torch.from_numpy(t).cuda()
    md = torch.from_numpy(mu).cuda()
    W = torch.empty_like(Hd)
    obj = torch.empty(B, device="cuda")
    res = torch.empty(B, device="cuda")
    fl = torch.empty(B, device="cuda", dtype=torch.int32)
    out = (W, obj, res, fl)
    stream = torch.cuda.current_stream()
    for _ in range(max(args.warmup, 3)):
        plan.solve(Hd, td, md, out=out)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            evs[i][0].record(stream)
            plan.solve(Hd, td, md, out=out)
            evs[i][1].record(stream)
        stop.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    total_ms = start.elapsed_time(stop)
    kern_ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    if world > 1:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / args.steps
    value = world * B / (ms_per_step / 1e3)
    clocks = clk.summary()
    props = torch.cuda.get_device_properties(local)
    max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    run_mhz = (clocks or {}).get("sm_mhz") or max_mhz
    set_fp32_peak(props.multi_processor_count, run_mhz,
                  f"{props.multi_processor_count} SMs (queried) x 128 FP32 lanes x 2 flop x "
                  f"{run_mhz:.0f} MHz (median SM clock sampled under load; maximum {max_mhz:.0f})")
    flags_np = fl.cpu().numpy()
    obj_np = obj.cpu().numpy()
    res_np = res.cpu().numpy()
    Wnp = W.cpu().numpy()

    # roofline of the solve kernel (FP32 FMA pipe)
    fpi = flops_per_instance(K, M, T, 1)
    achieved = fpi * B / (kern_ms / 1e3) / 1e12
    peak = fp32_peak_tflops()
    hbm_bytes = B * K * M * 8 * 2 + B * (K + 3) * 4
    peaks = measured_peaks()
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": "derived: " + _PEAK["source"],
            "kernel_ms": kern_ms,
            "flop_per_instance": fpi,
            "hbm": {"achieved_gbs": hbm_bytes / (kern_ms / 1e3) / 1e9,
                    "peak_gbs": peaks.get("hbm_gbs"), "algorithmic_bytes": hbm_bytes}}
    plan_kernel_name = capi.precode_plan_describe(plan.handle, M, K)
    roof["kernel"] = plan_kernel_name
    if plan_kernel_name.startswith("solve_tch_kernel"):
        # layers and setup as split FP16 (m16n8k16): issued MMA work as a share of the
        # dense tensor peaks (FP16 = the measured bf16 peak; TF32 = that times the
        # nominal ratio 1.1 / 2.25), summed as pipe time
        n16, n8 = mma_per_instance_f16(T)
        sec = kern_ms / 1e3
        i16 = n16 * 2 * 16 * 8 * 16 * B / sec / 1e12
        i8 = n8 * 2 * 16 * 8 * 8 * B / sec / 1e12
        f16_peak = peaks.get("bf16_tflops", 1900.0)
        tf32_peak = f16_peak * 1.1 / 2.25
        roof["tensor"] = {"mma_m16n8k16_f16_per_instance": n16, "mma_m16n8k8_tf32_per_instance": n8,
                          "issued_tflops": i16 + i8, "peak_f16_tflops": f16_peak,
                          "peak_tf32_tflops": tf32_peak, "frac": i16 / f16_peak + i8 / tf32_peak,
                          "peak_source": "of measured: bf16_tflops (FP16), x 1.1 / 2.25 (TF32)"}
    elif plan_kernel_name.startswith("solve_tc_kernel"):
        # the contractions run on the tensor cores as split TF32 (three MMAs per
        # FP32-accurate product): issued MMA work against the TF32 dense peak
        # (the measured bf16 peak times the nominal TF32 / bf16 ratio 1.1 / 2.25)
        mma = mma_per_instance(T)
        issued = mma * 2 * 16 * 8 * 8 * B / (kern_ms / 1e3) / 1e12
        tf32_peak = peaks.get("bf16_tflops", 1900.0) * 1.1 / 2.25
        roof["tensor"] = {"mma_m16n8k8_per_instance": mma, "issued_tflops": issued,
                          "peak_tf32_tflops": tf32_peak, "frac": issued / tf32_peak,
                          "peak_source": "of measured: bf16_tflops x 1.1 / 2.25"}
    # DRAM traffic per launch from a committed ncu capture, if one was taken on
    # the kernel variant that ran here
    import glob
    for prof in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.traffic.txt"))):
        kv = dict(line.split(": ", 1) for line in open(prof).read().splitlines() if ": " in line)
        if kv.get("kernel", "").strip() == plan_kernel_name:
            roof["traffic"] = int(kv["traffic_bytes_per_launch"])
            roof["traffic_source"] = kv.get("source")

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "fixed: 65,536 x C^{8x64} per GPU, CN(0,1) with 8 dB log-normal "
                                   "user gains, unit targets, T=10 projected layers, "
                                   "mu_t ~ U[0.01,0.1] (seed 2)",
                       "B_per_gpu": B, "K": K, "M": M, "T": T, "layer": "projected",
                       "l2": "inputs larger than L2 (268 MB of H per step), no flush",
                       "parallelism": f"independent shards x{world}"},
            "gpu_launches": args.steps, "roofline": roof, "clocks": clocks,
            "flags_nonzero": int((flags_np != 0).sum()),
            "fp64_fallbacks": int(((flags_np & capi.F_FP64_CHOL) != 0).sum())}

    # end to end through the C ABI with pinned host buffers
    Hh = torch.from_numpy(H).pin_memory()
    th = torch.from_numpy(t).pin_memory()
    mh = torch.from_numpy(mu)
    Wh = torch.empty_like(Hh).pin_memory()
    oh = torch.empty(B).pin_memory()
    rh = torch.empty(B).pin_memory()
    fh = torch.empty(B, dtype=torch.int32).pin_memory()
    plan.solve_host(Hh, th, mh, None, W=Wh, obj=oh, resid=rh, flags=fh)
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        plan.solve_host(Hh, th, mh, None, W=Wh, obj=oh, resid=rh, flags=fh)
    e2e_s = (time.perf_counter() - t0) / args.e2e_steps
    if world > 1:
        tt = torch.tensor([e2e_s], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_s = float(tt.item())
    h2d_b, d2h_b = int(H.nbytes + t.nbytes + 4 * T), int(H.nbytes + 3 * 4 * B)
    link = host_link_peak(torch)
    line["e2e"] = {"value": world * B / e2e_s, "unit": UNIT,
                   "h2d_bytes_per_step": h2d_b,
                   "d2h_bytes_per_step": d2h_b,
                   "host_link": link,
                   "host_link_frac": (h2d_b + d2h_b) / e2e_s / 1e9 / link["both_gbs"],
                   "host_link_frac_source": "bytes moved per step / step time, against the "
                                            "measured both-directions copy bandwidth",
                   "api": "precode_solve_host (pinned host buffers: the zero-copy kernel reads H and "
                          "writes W over the host link; pageable buffers would take the staged "
                          "copy pipeline)"}

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb, (lo, oobj) = cpu_baseline(H, t, mu)
        n = len(oobj)
        line["cpu_baseline"] = cb
        gap = np.abs(obj_np[lo:lo + n] - oobj) / oobj
        import oracle
        pcg = [oracle.pcg(H[b].astype(np.complex128), t[b].astype(np.float64),
                          Wnp[b].astype(np.complex128)) for b in range(lo, lo + min(n, 256))]
        line["pa_gap"] = {"rel_obj_diff_gpu_vs_oracle_max": float(gap.max()),
                          "rel_obj_diff_gpu_vs_oracle_mean": float(gap.mean()),
                          "rel_obj_diff_gpu_vs_oracle_p50": float(np.percentile(gap, 50)),
                          "rel_obj_diff_gpu_vs_oracle_p99": float(np.percentile(gap, 99)),
                          "instances": n, "mean_pcg_gpu": float(np.mean(pcg))}
    plan.close()
    del Hd, W
    if rank == 0 and not args.no_extras:
        from paper_2304_12745_gb300.precoder import inst_table
        torch.cuda.empty_cache()
        line["uneven"] = bench_uneven(torch, capi, Plan, inst_table)
        line["train"], mu_learned = bench_train(torch, capi)
        torch.cuda.empty_cache()
        line["serving"] = bench_serve(capi, mu_learned)
        line["serving"]["resident"] = bench_resident(capi, mu_learned)
        torch.cuda.empty_cache()
        line["paper_setting"] = bench_paper_setting(torch, capi)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
