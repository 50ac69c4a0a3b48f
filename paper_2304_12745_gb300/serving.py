"""Python handle on the library's continuous-batching server (argument marshalling).

``Server.submit`` takes numpy arrays (pinned copies are made once per job so the
host<->device copies can overlap); results land in the job's output arrays.
``poisson_load`` drives a server with Poisson arrivals of random jobs and
returns the server's latency statistics.
"""
from __future__ import annotations

import time

import numpy as np

from . import capi, channels


class JobHandle:
    def __init__(self, server, ticket, arrays):
        self.server, self.ticket, self.arrays = server, ticket, arrays
        self.result = None

    def wait(self, timeout_us: int = -1):
        if self.result is None:
            self.result = capi.precode_serve_wait(self.server.handle, self.ticket, timeout_us)
        return self.result

    @property
    def W(self):
        return self.arrays["W"]

    @property
    def obj(self):
        return self.arrays["obj"]

    @property
    def flags(self):
        return self.arrays["flags"]


class Server:
    def __init__(self, mode: int, step, lam=None, shapes=((64, 8),), *, n_slots: int = 4,
                 max_batch_instances: int = 16384, device_mem_budget: int = 0, device: int = 0,
                 cond_threshold: float = 0.0, flags: int = 0):
        self.step = np.ascontiguousarray(step, dtype=np.float32)
        self.lam = None if lam is None else np.ascontiguousarray(lam, dtype=np.float32)
        self.T = len(self.step)
        self.handle = capi.precode_serve_create(mode, self.T, self.step, self.lam, list(shapes),
                                                n_slots, max_batch_instances, device_mem_budget,
                                                device, cond_threshold, flags)

    def submit(self, H: np.ndarray | None, t: np.ndarray, *, channel: int = 0, M=None, K=None,
               n_sc=None) -> JobHandle:
        if H is not None:
            n_sc, K, M = H.shape
            H = np.ascontiguousarray(H, dtype=np.complex64)
        t = np.ascontiguousarray(t, dtype=np.float32)
        arrays = {"H": H, "t": t, "W": np.empty((n_sc, K, M), np.complex64),
                  "obj": np.empty(n_sc, np.float32), "resid": np.empty(n_sc, np.float32),
                  "flags": np.empty(n_sc, np.int32)}
        job = capi.Job(M, K, n_sc, capi.ptr(H), capi.ptr(t), 1 if t.ndim == 1 else 0,
                       capi.ptr(arrays["W"]), capi.ptr(arrays["obj"]), capi.ptr(arrays["resid"]),
                       capi.ptr(arrays["flags"]), channel)
        return JobHandle(self, capi.precode_serve_submit(self.handle, job), arrays)

    def channel(self, H: np.ndarray) -> int:
        n_sc, K, M = H.shape
        H = np.ascontiguousarray(H, dtype=np.complex64)
        return capi.precode_serve_channel_create(self.handle, M, K, n_sc, H)

    def release_channel(self, handle: int):
        capi.precode_serve_channel_destroy(self.handle, handle)

    def stats(self) -> dict:
        s = capi.precode_serve_stats(self.handle)
        return {f: getattr(s, f) for f, _ in s._fields_}

    def reset_stats(self):
        capi.precode_serve_reset_stats(self.handle)

    def close(self):
        if self.handle:
            capi.precode_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def pinned(n: int, dtype) -> np.ndarray:
    """Page-locked host array (lets the server's copies run asynchronously)."""
    import torch
    tdt = {np.complex64: torch.complex64, np.float32: torch.float32}[dtype]
    return torch.empty(n, dtype=tdt, pin_memory=True).numpy()


def touch_by_device(*arrays: np.ndarray, chunk_bytes: int = 256 << 20):
    """Read each page-locked array into device memory and write it back, chunk by
    chunk: the device's first access to a page of host memory sets up its address
    translation, and that cost would otherwise land on the first jobs that use the
    page (a latency spike of tens of ms on a fresh 4 GB output ring)."""
    import torch
    dev = torch.empty(chunk_bytes, dtype=torch.uint8, device="cuda")
    for a in arrays:
        flat = torch.from_numpy(a.reshape(-1).view(np.uint8))
        for lo in range(0, flat.numel(), chunk_bytes):
            part = flat[lo:lo + chunk_bytes]
            d = dev[:part.numel()]
            d.copy_(part, non_blocking=True)
            part.copy_(d, non_blocking=True)
    torch.cuda.synchronize()


def random_job(rng: np.random.Generator, M_choices=(64, 128, 256), K_range=(4, 32),
               nsc_choices=(64, 128, 256, 512, 1024)):
    M = int(rng.choice(M_choices))
    K = int(rng.integers(K_range[0], min(K_range[1], M) + 1))
    n_sc = int(rng.choice(nsc_choices))
    return M, K, n_sc


def poisson_load(server: Server, rate_per_s: float, duration_s: float, seed: int,
                 M_choices=(64, 128, 256), K_range=(4, 32), nsc_choices=(64, 128, 256, 512, 1024),
                 ring_bytes: int = 4 << 30) -> dict:
    """Submit jobs with exponential inter-arrival times for `duration_s`, wait for
    all, return the server's statistics.

    Inputs come from one pre-generated pool of Rician channels (a job's H is the
    first n_sc*K*M values of the pool, viewed as [n_sc][K][M]), so generation stays
    off the clock; outputs go to slices of a host ring buffer that is reused only
    after the job that held a slice finished.  Both are touched by the device once
    before the clock starts, as a long-running caller's buffers would be."""
    rng = np.random.default_rng(seed)
    n_max = max(nsc_choices) * K_range[1] * max(M_choices)
    pool = pinned(n_max, np.complex64)
    pool[:] = channels.rician_ula(1, 1, n_max, seed=seed)[0, 0]
    ring = pinned(ring_bytes // 8, np.complex64)
    ones = pinned(K_range[1], np.float32)
    ones[:] = 1.0
    touch_by_device(pool, ring, ones)
    sched, t = [], 0.0
    while t < duration_s:
        t += rng.exponential(1.0 / rate_per_s)
        sched.append((t,) + random_job(rng, M_choices, K_range, nsc_choices))
    server.reset_stats()
    handles, live, cursor = [], [], 0
    t0 = time.perf_counter()
    for at, M, K, n_sc in sched:
        n = n_sc * K * M
        if cursor + n > ring.size:
            cursor = 0
        # the ring slice must be free: wait for every live job overlapping it
        while live and any(lo < cursor + n and cursor < hi for lo, hi, _ in live):
            lo, hi, h = live.pop(0)
            h.wait()
        while time.perf_counter() - t0 < at:
            pass
        H = pool[:n].reshape(n_sc, K, M)
        W = ring[cursor:cursor + n].reshape(n_sc, K, M)
        arrays = {"H": H, "t": ones, "W": W, "obj": np.empty(n_sc, np.float32),
                  "resid": None, "flags": np.empty(n_sc, np.int32)}
        job = capi.Job(M, K, n_sc, capi.ptr(H), capi.ptr(ones), 1, capi.ptr(W),
                       capi.ptr(arrays["obj"]), None, capi.ptr(arrays["flags"]), 0)
        h = JobHandle(server, capi.precode_serve_submit(server.handle, job), arrays)
        handles.append(h)
        live.append((cursor, cursor + n, h))
        cursor += n
    for h in handles:
        h.wait()
    wall = time.perf_counter() - t0
    st = server.stats()
    st["jobs"] = len(handles)
    st["offered_rate_per_s"] = rate_per_s
    st["achieved_rate_per_s"] = len(handles) / wall
    return st
