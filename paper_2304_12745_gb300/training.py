"""Learning the per-layer parameters (Sec. V): autograd bridge and Adam trainer.

``PrecodeLoss`` is a ``torch.autograd.Function`` whose forward calls the
library's ``precode_train_step`` (forward + adjoint kernels in one go) and keeps
the parameter gradients for ``backward``.  ``UnfoldedTrainer`` runs Adam on the
per-layer parameters over batches of synthetic channels and applies the paper's
parameter projections after every step:

* paper layer:     lambda <- max(0, lambda), eta <- min(max(eta, 1/(2 L~)), 1/L~),
                   L~ = (sqrt K + sqrt M)^2 (Marchenko-Pastur edge);
* projected layer: mu <- max(0, mu).

The unsupervised cost is a ||W_T||_{2,1} + ||H W_T^T - S||_F^2 averaged over the
batch (a = lambda in the paper's cost; the PA-consumption weight for the
projected layer).  The supervised cost (labels given) is the MSE
||W_T - W_gt||_F^2 to ground-truth precoders, averaged over the batch.
"""
from __future__ import annotations

import math

import torch

from . import capi, channels
from .precoder import Plan, _stream_handle


class PrecodeLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, step, lam, plan, H, t, a, group=None, labels=None):
        B, K, M = H.shape
        dev = H.device
        loss = torch.empty(1, device=dev)
        dstep = torch.empty_like(step)
        dlam = torch.empty_like(step) if lam is not None else None
        t_stride = 0 if t.dim() == 1 else K
        lm = None if lam is None else lam.detach().contiguous()
        if labels is None:
            capi.precode_train_step(plan.handle, M, K, B, H, t, t_stride, step.detach().contiguous(),
                                    lm, a, loss, dstep, dlam, None, _stream_handle(None))
        else:
            assert labels.shape == H.shape and labels.dtype == torch.complex64 and labels.is_cuda
            capi.precode_train_step_supervised(plan.handle, M, K, B, H, t, t_stride,
                                               labels.contiguous(), step.detach().contiguous(), lm,
                                               loss, dstep, dlam, None, _stream_handle(None))
        if group is not None:  # data-parallel ranks: global batch mean (2T + 2 numbers)
            from .sharding import allreduce_mean
            loss, dstep, dlam = allreduce_mean(loss, dstep, dlam, B, group)
        ctx.save_for_backward(dstep, dlam if dlam is not None else dstep)
        ctx.has_lam = lam is not None
        return loss.reshape(-1)[0]

    @staticmethod
    def backward(ctx, g):
        dstep, dlam = ctx.saved_tensors
        return g * dstep, (g * dlam if ctx.has_lam else None), None, None, None, None, None, None


def mp_bound(K: int, M: int) -> float:
    """L~ = (sqrt K + sqrt M)^2."""
    return (math.sqrt(K) + math.sqrt(M)) ** 2


class UnfoldedTrainer:
    """Adam over the per-layer parameters of one layer map on one (M, K)."""

    MAX_GRAPHS = 16  # captured steps kept with graphs=True (one per resident batch)

    def __init__(self, mode: int, T: int, K: int, M: int, batch: int, *, a: float,
                 lr: float = 1e-3, init_step=None, init_lam=None, device: str = "cuda",
                 step_normalised: bool = False, group=None, tensor_cores: bool = True,
                 graphs: bool = False):
        """`group`: a torch.distributed process group whose ranks each train on
        their own batches; gradients are averaged over all ranks every step.
        `tensor_cores`: use the tensor-core forward + adjoint build where the
        shape has one (K = 8, M = 64: split FP16 for the projected layer, split
        TF32 for the paper layer).
        `graphs`: replay each step (forward + adjoint launch, batch reduction,
        backward, Adam, projection) as one CUDA graph per resident batch: the
        first step on a batch runs eagerly and captures the graph, later steps on
        the same (H, t) tensors replay it.  Single-process trainers only."""
        if graphs and group is not None:
            raise ValueError("graphs=True needs a single-process trainer (group=None)")
        self.mode, self.T, self.K, self.M, self.batch, self.a = mode, T, K, M, batch, a
        self.group = group
        self.graphs = graphs
        self._graphs = {}
        self.plan = Plan(mode, T, [(M, K)], batch, step_normalised=step_normalised,
                         tensor_cores=tensor_cores)
        L = mp_bound(K, M)
        if init_step is None:
            init_step = [1.0 / L] * T if mode == capi.LAYER_PGD else [0.05] * T
        self.step = torch.nn.Parameter(torch.tensor(init_step, dtype=torch.float32, device=device))
        params = [self.step]
        self.lam = None
        if mode == capi.LAYER_PGD:
            init_lam = [1.0 / 15] * T if init_lam is None else init_lam
            self.lam = torch.nn.Parameter(torch.tensor(init_lam, dtype=torch.float32,
                                                       device=device))
            params.append(self.lam)
        # one fused kernel per optimiser step on CUDA parameters; with graphs the
        # step count lives on the device so that the captured update can advance it
        self.opt = torch.optim.Adam(params, lr=lr, fused=self.step.is_cuda, capturable=graphs)
        self.steps_done = 0

    def project(self):
        """Parameter projections after each optimiser step (Sec. V end)."""
        with torch.no_grad():
            if self.mode == capi.LAYER_PGD:
                L = mp_bound(self.K, self.M)
                self.lam.clamp_(min=0.0)
                self.step.clamp_(min=1.0 / (2 * L), max=1.0 / L)
            else:
                self.step.clamp_(min=0.0)

    def loss(self, H: torch.Tensor, t: torch.Tensor, labels=None) -> torch.Tensor:
        return PrecodeLoss.apply(self.step, self.lam, self.plan, H, t, self.a, self.group, labels)

    def train_step(self, H: torch.Tensor, t: torch.Tensor, sync: bool = True, labels=None):
        """One Adam step on batch (H, t).  Returns the batch loss as a float, or
        with sync=False as a device tensor (no host synchronisation, so steps
        queue back to back on the stream).  `labels` (complex64 [B, K, M] on the
        device): ground-truth precoders for the supervised cost instead of the
        unsupervised one."""
        if self.graphs:
            loss = self._graphed_step(H, t, labels)
        else:
            loss = self._eager_step(H, t, labels)
        self.steps_done += 1
        return float(loss) if sync else loss

    def _eager_step(self, H: torch.Tensor, t: torch.Tensor, labels=None) -> torch.Tensor:
        self.opt.zero_grad(set_to_none=True)
        loss = self.loss(H, t, labels)
        loss.backward()
        self.opt.step()
        self.project()
        return loss.detach()

    def _graphed_step(self, H: torch.Tensor, t: torch.Tensor, labels=None) -> torch.Tensor:
        key = (H.data_ptr(), tuple(H.shape), t.data_ptr(), tuple(t.shape),
               None if labels is None else labels.data_ptr())
        entry = self._graphs.get(key)
        if entry is not None:
            graph, loss = entry
            graph.replay()
            return loss.clone()
        # First step on this batch: a real eager step (it also sizes the plan's
        # workspace and settles the optimiser state), then the capture of the
        # same step, which records the work without running it.  At most
        # MAX_GRAPHS batches keep a graph (the oldest is dropped): a caller that
        # brings a new tensor every step gets eager steps plus a capture each time,
        # so graphs pay off only for batches that stay resident.
        loss = self._eager_step(H, t, labels)
        if len(self._graphs) >= self.MAX_GRAPHS:
            self._graphs.pop(next(iter(self._graphs)))
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        self.opt.zero_grad(set_to_none=True)
        with torch.cuda.graph(graph):
            static_loss = self.loss(H, t, labels)
            static_loss.backward()
            self.opt.step()
            self.project()
        self._graphs[key] = (graph, static_loss.detach())
        return loss

    def make_batch(self, index: int, seed: int, family: str = "rayleigh"):
        """Channels of batch `index` (deterministic in (seed, index))."""
        H = channels.channels(family, self.batch, self.K, self.M, seed=seed * 1000003 + index)
        return torch.from_numpy(H).to(self.step.device)

    def state_dict(self):
        return {"step": self.step.detach().clone(),
                "lam": None if self.lam is None else self.lam.detach().clone(),
                "opt": self.opt.state_dict(), "steps_done": self.steps_done}

    def load_state_dict(self, s):
        with torch.no_grad():
            self.step.copy_(s["step"])
            if self.lam is not None:
                self.lam.copy_(s["lam"])
        self.opt.load_state_dict(s["opt"])
        self.steps_done = s["steps_done"]
        self._graphs.clear()  # captured steps refer to the replaced optimiser state
