"""Torch-facing wrapper of the C ABI (plans and batched solves).

Only argument marshalling lives here: shapes are checked, output tensors are
allocated with torch, and the library's entry points are called with their
addresses and the current CUDA stream.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def inst_table(h_off, w_off, t_off, M, K) -> torch.Tensor:
    """Pack per-instance descriptors (``precode_inst_t``: three int64 offsets, then
    int32 M and K) into an int64 tensor [B, 4] on the CPU."""
    dt = np.dtype([("h", "<i8"), ("w", "<i8"), ("t", "<i8"), ("M", "<i4"), ("K", "<i4")])
    h_off = np.asarray(h_off, dtype=np.int64).reshape(-1)
    a = np.zeros(h_off.size, dt)
    a["h"], a["w"], a["t"] = h_off, np.asarray(w_off).reshape(-1), np.asarray(t_off).reshape(-1)
    a["M"], a["K"] = np.asarray(M).reshape(-1), np.asarray(K).reshape(-1)
    return torch.from_numpy(a.view(np.int64).reshape(h_off.size, 4).copy())


class Plan:
    """A ``precode_plan_t``: layer map, T, shapes, kernel choice and workspace."""

    def __init__(self, mode: int, T: int, shapes, max_instances: int, *,
                 cond_threshold: float = 0.0, autotune: bool = False,
                 step_normalised: bool = False, graphs: bool = False,
                 tensor_cores: bool = False, device: int | None = None,
                 tune_cache: str | None = None):
        if device is None:
            device = torch.cuda.current_device()
        flags = (capi.PLAN_AUTOTUNE if autotune else 0) | \
                (capi.PLAN_STEP_NORMALISED if step_normalised else 0) | \
                (capi.PLAN_GRAPHS if graphs else 0) | \
                (capi.PLAN_TENSOR_CORES if tensor_cores else 0)
        self.mode, self.T, self.device = mode, T, device
        self.shapes = [tuple(s) for s in shapes]
        self.max_instances = max_instances
        self.handle = capi.precode_plan(mode, T, self.shapes, max_instances, cond_threshold, flags,
                                        device, tune_cache)

    def close(self):
        if self.handle:
            capi.precode_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, H: torch.Tensor, t: torch.Tensor, step: torch.Tensor,
              lam: torch.Tensor | None = None, *, want_obj: bool = True, want_resid: bool = True,
              want_flags: bool = True, out=None, stream=None):
        """Batched solve of H [B, K, M] complex64 (device).  t: [B, K] or [K] float32.
        step / lam: float32 [T] on the device.  Returns (W, obj, resid, flags)."""
        assert H.is_cuda and H.dtype == torch.complex64 and H.dim() == 3 and H.is_contiguous()
        B, K, M = H.shape
        assert t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
        t_stride = 0 if t.dim() == 1 else K
        assert step.is_cuda and step.dtype == torch.float32 and step.numel() == self.T
        if lam is not None:
            assert lam.is_cuda and lam.dtype == torch.float32 and lam.numel() == self.T
        dev = H.device
        if out is None:
            W = torch.empty_like(H)
            obj = torch.empty(B, device=dev, dtype=torch.float32) if want_obj else None
            resid = torch.empty(B, device=dev, dtype=torch.float32) if want_resid else None
            flags = torch.empty(B, device=dev, dtype=torch.int32) if want_flags else None
        else:
            W, obj, resid, flags = out
        capi.precode_solve(self.handle, M, K, B, H, t, t_stride, step, lam, W, obj, resid, flags,
                           _stream_handle(stream))
        return W, obj, resid, flags

    def solve_varlen(self, tbl: torch.Tensor, H: torch.Tensor, t: torch.Tensor, step: torch.Tensor,
                     lam: torch.Tensor | None = None, *, W: torch.Tensor | None = None,
                     want_resid: bool = True, stream=None):
        """Uneven batch: ``tbl`` is the device int64 [B, 4] descriptor table
        (see ``inst_table``), H / W flat complex64 buffers holding every instance,
        t a flat float32 buffer.  Returns (W, obj, resid, flags)."""
        assert tbl.is_cuda and tbl.dtype == torch.int64 and tbl.dim() == 2 and tbl.shape[1] == 4
        B = tbl.shape[0]
        dev = H.device
        W = torch.empty_like(H) if W is None else W
        obj = torch.empty(B, device=dev, dtype=torch.float32)
        resid = torch.empty(B, device=dev, dtype=torch.float32) if want_resid else None
        flags = torch.zeros(B, device=dev, dtype=torch.int32)
        capi.precode_solve_varlen(self.handle, B, tbl, H, t, step, lam, W, obj, resid, flags,
                                  _stream_handle(stream))
        return W, obj, resid, flags

    def solve_host(self, H, t, step, lam=None, *, W=None, obj=None, resid=None, flags=None):
        """Same computation from host (CPU, ideally pinned) tensors; synchronous."""
        B, K, M = H.shape
        t_stride = 0 if t.dim() == 1 else K
        W = torch.empty_like(H) if W is None else W
        capi.precode_solve_host(self.handle, M, K, B, H, t, t_stride, step, lam, W, obj, resid,
                                flags)
        return W, obj, resid, flags

    def errors(self) -> int:
        return capi.precode_plan_errors(self.handle)
