"""ctypes binding of ``libprecode.so`` -- argument marshalling only.

Every function here has the name of the C entry point it calls and forwards
plain pointers and sizes; the computation runs in the library's CUDA kernels.
There is no CPU fallback: if the library is missing or fails to load, the
import raises.  Tensors are torch tensors used only as device (or pinned host)
memory; their ``data_ptr()`` is what crosses the boundary.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libprecode.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEDOUT, EBUSY, PENDING, ENOTFOUND = range(8)
LAYER_PGD, LAYER_PROJ = 0, 1
F_FP64_CHOL, F_SINGULAR, F_NONFINITE, F_TIMEOUT, F_INVALID = 1, 2, 4, 8, 16
PLAN_AUTOTUNE, PLAN_STEP_NORMALISED, PLAN_GRAPHS, PLAN_TENSOR_CORES = 1, 2, 4, 8
MAX_K, MAX_M, MAX_T = 32, 256, 65536


class PrecodeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class Shape(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("K", ctypes.c_int32)]


class Desc(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("T", ctypes.c_int32), ("n_shapes", ctypes.c_int32),
                ("shapes", ctypes.POINTER(Shape)), ("max_instances", ctypes.c_int64),
                ("cond_threshold", ctypes.c_double), ("flags", ctypes.c_uint32),
                ("device", ctypes.c_int32), ("tune_cache", ctypes.c_char_p)]


class ServeDesc(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("T", ctypes.c_int32),
                ("step", ctypes.c_void_p), ("lam", ctypes.c_void_p),
                ("n_shapes", ctypes.c_int32), ("shapes", ctypes.POINTER(Shape)),
                ("n_slots", ctypes.c_int32), ("max_batch_instances", ctypes.c_int64),
                ("device_mem_budget", ctypes.c_int64), ("device", ctypes.c_int32),
                ("cond_threshold", ctypes.c_double), ("flags", ctypes.c_uint32)]


class Job(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int32), ("K", ctypes.c_int32), ("n_sc", ctypes.c_int32),
                ("H", ctypes.c_void_p), ("t", ctypes.c_void_p), ("t_shared", ctypes.c_int32),
                ("W_out", ctypes.c_void_p), ("obj_out", ctypes.c_void_p),
                ("resid_out", ctypes.c_void_p), ("flags_out", ctypes.c_void_p),
                ("channel", ctypes.c_uint64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("submit_us", ctypes.c_double),
                ("start_us", ctypes.c_double), ("done_us", ctypes.c_double),
                ("latency_us", ctypes.c_double)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("rejected", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double),
                ("max_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("precoders_per_s", ctypes.c_double), ("instances_done", ctypes.c_int64),
                ("bytes_in_use", ctypes.c_int64), ("bytes_budget", ctypes.c_int64),
                ("slots_busy", ctypes.c_int32), ("queued", ctypes.c_int32),
                ("factor_instances", ctypes.c_int64)]


_vp = ctypes.c_void_p
_i32, _i64, _u32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32

_SIGS = {
    "precode_plan": [ctypes.POINTER(Desc), ctypes.POINTER(_vp)],
    "precode_plan_destroy": [_vp],
    "precode_solve": [_vp, _i32, _i32, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "precode_solve_host": [_vp, _i32, _i32, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp],
    "precode_plan_errors": [_vp, ctypes.POINTER(ctypes.c_uint64)],
    "precode_plan_set_debug": [_vp, ctypes.c_uint64, _i32],
    "precode_plan_describe": [_vp, _i32, _i32, ctypes.c_char_p, ctypes.c_size_t],
    "precode_solve_varlen": [_vp, _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "precode_train_step": [_vp, _i32, _i32, _i64, _vp, _vp, _i64, _vp, _vp, ctypes.c_float, _vp,
                           _vp, _vp, _vp, _vp],
    "precode_train_step_supervised": [_vp, _i32, _i32, _i64, _vp, _vp, _i64, _vp, _vp, _vp, _vp,
                                      _vp, _vp, _vp, _vp],
    "precode_serve_create": [ctypes.POINTER(ServeDesc), ctypes.POINTER(_vp)],
    "precode_serve_submit": [_vp, ctypes.POINTER(Job), ctypes.POINTER(ctypes.c_uint64)],
    "precode_serve_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(Result)],
    "precode_serve_wait": [_vp, ctypes.c_uint64, _i64, ctypes.POINTER(Result)],
    "precode_serve_stats": [_vp, ctypes.POINTER(ServeStats)],
    "precode_serve_reset_stats": [_vp],
    "precode_serve_channel_create": [_vp, _i32, _i32, _i32, _vp, ctypes.POINTER(ctypes.c_uint64)],
    "precode_serve_channel_destroy": [_vp, ctypes.c_uint64],
    "precode_serve_destroy": [_vp],
    "precode_solve_varlen_static": [ctypes.POINTER(Desc), _i64, _vp, _vp, _vp, _vp, _vp, _vp, _vp,
                                    _vp, _vp, _vp],
}


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2304_12745_gb300.build` "
            "(or __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.precode_status_str.argtypes = [ctypes.c_int]
    lib.precode_status_str.restype = ctypes.c_char_p
    lib.precode_last_error.argtypes = []
    lib.precode_last_error.restype = ctypes.c_char_p
    return lib


LIB = _load()


def check(status: int, where: str):
    if status != OK:
        raise PrecodeError(status, where, LIB.precode_last_error().decode(errors="replace")
                           or LIB.precode_status_str(status).decode())


def ptr(x) -> int | None:
    """Device (or host) address of a tensor / numpy array, None for None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def precode_plan(mode: int, T: int, shapes, max_instances: int, cond_threshold: float = 0.0,
                 flags: int = 0, device: int = 0, tune_cache: str | None = None) -> int:
    arr = (Shape * len(shapes))(*[Shape(int(m), int(k)) for (m, k) in shapes])
    d = Desc(mode, T, len(shapes), arr, max_instances, cond_threshold, flags, device,
             tune_cache.encode() if tune_cache else None)
    h = _vp()
    check(LIB.precode_plan(ctypes.byref(d), ctypes.byref(h)), "precode_plan")
    return h.value


def precode_plan_destroy(plan: int):
    check(LIB.precode_plan_destroy(plan), "precode_plan_destroy")


def precode_solve(plan, M, K, B, H, t, t_stride, step, lam, W, obj, resid, flags, stream):
    check(LIB.precode_solve(plan, M, K, B, ptr(H), ptr(t), t_stride, ptr(step), ptr(lam), ptr(W),
                            ptr(obj), ptr(resid), ptr(flags), stream), "precode_solve")


def precode_solve_host(plan, M, K, B, H, t, t_stride, step, lam, W, obj, resid, flags):
    check(LIB.precode_solve_host(plan, M, K, B, ptr(H), ptr(t), t_stride, ptr(step), ptr(lam),
                                 ptr(W), ptr(obj), ptr(resid), ptr(flags)), "precode_solve_host")


def precode_solve_varlen(plan, B, tbl, H, t, step, lam, W, obj, resid, flags, stream):
    check(LIB.precode_solve_varlen(plan, B, ptr(tbl), ptr(H), ptr(t), ptr(step), ptr(lam), ptr(W),
                                   ptr(obj), ptr(resid), ptr(flags), stream), "precode_solve_varlen")


def precode_solve_varlen_static(mode, T, shapes, B, tbl, H, t, step, lam, W, obj, resid, flags,
                                stream, cond_threshold: float = 0.0, flags_desc: int = 0,
                                device: int = 0):
    """Uneven batch without a plan; the library's fixed scratch array is used."""
    arr = (Shape * len(shapes))(*[Shape(int(m), int(k)) for (m, k) in shapes])
    d = Desc(mode, T, len(shapes), arr, 0, cond_threshold, flags_desc, device, None)
    check(LIB.precode_solve_varlen_static(ctypes.byref(d), B, ptr(tbl), ptr(H), ptr(t), ptr(step),
                                          ptr(lam), ptr(W), ptr(obj), ptr(resid), ptr(flags),
                                          stream), "precode_solve_varlen_static")


def precode_train_step(plan, M, K, B, H, t, t_stride, step, lam, a, loss, dstep, dlam, flags,
                       stream):
    check(LIB.precode_train_step(plan, M, K, B, ptr(H), ptr(t), t_stride, ptr(step), ptr(lam),
                                 float(a), ptr(loss), ptr(dstep), ptr(dlam), ptr(flags), stream),
          "precode_train_step")


def precode_train_step_supervised(plan, M, K, B, H, t, t_stride, W_gt, step, lam, loss, dstep,
                                  dlam, flags, stream):
    check(LIB.precode_train_step_supervised(plan, M, K, B, ptr(H), ptr(t), t_stride, ptr(W_gt),
                                            ptr(step), ptr(lam), ptr(loss), ptr(dstep), ptr(dlam),
                                            ptr(flags), stream), "precode_train_step_supervised")


def precode_serve_create(mode, T, step, lam, shapes, n_slots=4, max_batch_instances=16384,
                         device_mem_budget=0, device=0, cond_threshold=0.0, flags=0) -> int:
    arr = (Shape * len(shapes))(*[Shape(int(m), int(k)) for (m, k) in shapes])
    d = ServeDesc(mode, T, ptr(step), ptr(lam), len(shapes), arr, n_slots, max_batch_instances,
                  device_mem_budget, device, cond_threshold, flags)
    h = _vp()
    check(LIB.precode_serve_create(ctypes.byref(d), ctypes.byref(h)), "precode_serve_create")
    return h.value


def precode_serve_submit(server, job: Job) -> int:
    tk = ctypes.c_uint64(0)
    check(LIB.precode_serve_submit(server, ctypes.byref(job), ctypes.byref(tk)),
          "precode_serve_submit")
    return tk.value


def precode_serve_poll(server, ticket):
    r = Result()
    st = LIB.precode_serve_poll(server, ticket, ctypes.byref(r))
    if st == PENDING:
        return None
    check(st, "precode_serve_poll")
    return r


def precode_serve_wait(server, ticket, timeout_us=-1):
    r = Result()
    check(LIB.precode_serve_wait(server, ticket, timeout_us, ctypes.byref(r)), "precode_serve_wait")
    return r


def precode_serve_stats(server) -> ServeStats:
    s = ServeStats()
    check(LIB.precode_serve_stats(server, ctypes.byref(s)), "precode_serve_stats")
    return s


def precode_serve_reset_stats(server):
    check(LIB.precode_serve_reset_stats(server), "precode_serve_reset_stats")


def precode_serve_channel_create(server, M, K, n_sc, H) -> int:
    h = ctypes.c_uint64(0)
    check(LIB.precode_serve_channel_create(server, M, K, n_sc, ptr(H), ctypes.byref(h)),
          "precode_serve_channel_create")
    return h.value


def precode_serve_channel_destroy(server, handle):
    check(LIB.precode_serve_channel_destroy(server, handle), "precode_serve_channel_destroy")


def precode_serve_destroy(server):
    check(LIB.precode_serve_destroy(server), "precode_serve_destroy")


def precode_plan_describe(plan, M, K) -> str:
    buf = ctypes.create_string_buffer(256)
    check(LIB.precode_plan_describe(plan, M, K, buf, 256), "precode_plan_describe")
    return buf.value.decode()


def precode_plan_errors(plan) -> int:
    n = ctypes.c_uint64(0)
    check(LIB.precode_plan_errors(plan, ctypes.byref(n)), "precode_plan_errors")
    return n.value


def precode_plan_set_debug(plan, wait_limit_ns: int, inject_copy_stall: bool):
    check(LIB.precode_plan_set_debug(plan, int(wait_limit_ns), 1 if inject_copy_stall else 0),
          "precode_plan_set_debug")
