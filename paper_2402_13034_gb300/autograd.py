"""Differentiable RIS objective: J_b = sum over target receivers of log P_b(r) (Eq. 9, Eq. 10) as a
function of the element phases, with the hand-written adjoint of risrt_grad_phases as its backward,
and a gradient-ascent driver for RIS configuration."""
from __future__ import annotations

import torch


class RISLogPower(torch.autograd.Function):
    """phases [B, M] float32 CUDA -> J [B]; backward returns dJ/dphases from the adjoint kernel."""

    @staticmethod
    def forward(ctx, phases, objective):
        phases = phases.detach().contiguous()
        B, M = phases.shape
        J = torch.empty(B, dtype=torch.float32, device=phases.device)
        grad = torch.empty((B, M), dtype=torch.float32, device=phases.device)
        ws = objective.workspace(B)
        keep = objective.precision == 2 and objective._packed.get(B, False)   # A was packed by an earlier call
        # steps that reuse the packed A only enqueue (no synchronisation) when the library runs on torch's
        # current stream, which orders J and the gradient before torch reads them; check() reads the
        # tensor cores' timeout flag afterwards
        defer = keep and objective.lib.stream == torch.cuda.current_stream(phases.device).cuda_stream
        objective.lib.grad_phases(objective.A, objective.E0, objective.target, phases, objective.amp, J, grad,
                                  ws, objective.precision, keep_a=keep, defer_check=defer)
        objective._packed[B] = True
        ctx.save_for_backward(grad)
        return J

    @staticmethod
    def backward(ctx, gJ):
        (grad,) = ctx.saved_tensors
        return gJ[:, None] * grad, None


class PhaseObjective:
    """Binds a channel matrix A [n_rx, M] (complex64), E0 [n_rx], target rows (int32) and element
    amplitudes to the differentiable objective. They must not change while the objective is in use:
    the tensor-core path packs A once per workspace and reuses it."""

    def __init__(self, lib_ctx, A, E0=None, target=None, amp=None, precision=0):
        self.lib, self.A, self.E0, self.target, self.amp = lib_ctx, A, E0, target, amp
        self.precision = precision      # 0: FP32 CUDA cores, 2: split-BF16 tensor cores
        self._ws = {}
        self._packed = {}               # per B: the workspace holds A packed for the tensor-core path

    def workspace(self, B: int):
        if B not in self._ws:
            n_t = self.target.numel() if self.target is not None else self.A.shape[0]
            self._ws[B] = self.lib.grad_workspace(n_t, B, self.A.shape[1], self.precision)
        return self._ws[B]

    def __call__(self, phases):
        return RISLogPower.apply(phases, self)

    def check(self):
        """Raises RisrtError if a deferred tensor-core step of this objective timed out (waits for the stream)."""
        if self.precision == 2:
            for ws in self._ws.values():
                self.lib.grad_check(ws)


def ascend(objective: PhaseObjective, phases0, steps: int = 200, lr: float = 0.05):
    """Adam ascent on every configuration's phases at once; returns (phases, J per step [steps+1, B])."""
    phases = phases0.detach().clone().requires_grad_(True)
    opt = torch.optim.Adam([phases], lr=lr, maximize=True)
    hist = []
    for _ in range(steps):
        opt.zero_grad(set_to_none=True)
        J = objective(phases)
        J.sum().backward()
        hist.append(J.detach())
        opt.step()
    with torch.no_grad():
        hist.append(objective(phases).detach())
    objective.check()
    return phases.detach(), torch.stack(hist)
