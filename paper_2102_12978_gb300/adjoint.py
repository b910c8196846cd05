"""Gradient of a beam-quality loss with respect to the antenna weights.

`BeamLoss` is a torch.autograd.Function: its forward runs the Bessel-antenna
FDTD (library kernels) for `steps` steps with per-column amplitude / phase
weights on the annulus, saving the full state every `checkpoint` steps, and
averages the squared dominant E component at the probe points over the last
`window` steps (the time-averaged intensity of that component).  The loss is
the relative L2 distance of that map to a target map (for example
a J_0^2(K r) on the central lobes).  Its backward replays each checkpoint
segment forward to recover the probe values, and runs the library's
reverse-time adjoint through the segment, injecting dL/dE at the probes.

The steps before the loss window run as plain multi-step calls (any tile
configuration); the window's steps run through fdtd_probe_record, which
queues each step and its probe gather on the device without returning to
Python per step.  One grid, its adjoint and a zeroed initial state are made
per problem on first use and reused by every later forward and backward.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import torch

from . import fdtd


@dataclass
class BeamProblem:
    desc: fdtd.fdtd_grid_desc
    source: dict              # keyword arguments of Grid.set_source without the weights
    component: int            # E component read by the loss (FDTD_EX / FDTD_EY)
    probes: np.ndarray        # linear cell indices (k*ny + j)*nx + i
    target: torch.Tensor      # target intensity at the probes (device, float64)
    steps: int
    window: int
    checkpoint: int = 250
    tile: tuple | None = None     # tile configuration of the steps outside the loss window
    _ctx: dict = field(default_factory=dict, repr=False)

    def context(self):
        """(grid, adjoint, state at step 0) of this problem, made on first use."""
        if not self._ctx:
            grid = fdtd.Grid(self.desc)
            if self.tile is not None:
                grid.set_tile(*self.tile)
            grid.set_source(**self.source)
            adj = fdtd.Adjoint(grid, self.component, self.probes)
            self._ctx.update(grid=grid, adj=adj, zero=grid.save_state())
        return self._ctx["grid"], self._ctx["adj"], self._ctx["zero"]


def _set_weights(grid, prob: BeamProblem, w_amp: np.ndarray, w_phase: np.ndarray):
    grid.set_source(w_amp=w_amp, w_phase=w_phase, **prob.source)


def _run_forward(grid, adj, steps, record_from):
    """Step `steps` times; return the probe rows (device tensor, one row per
    step) of the steps whose output index (1-based, counted from the grid's
    step at entry) is >= record_from."""
    n0 = grid.n
    plain = max(0, min(steps, record_from - 1 - n0))
    if plain:
        grid.step(plain)
    return adj.record(steps - plain)


class BeamLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w_amp: torch.Tensor, w_phase: torch.Tensor, prob: BeamProblem):
        grid, adj, zero = prob.context()
        wa = w_amp.detach().double().cpu().numpy()
        wp = w_phase.detach().double().cpu().numpy()
        grid.load_state(zero)
        _set_weights(grid, prob, wa, wp)
        first = prob.steps - prob.window + 1          # window = E^first .. E^steps
        ckpts = {}
        rows = []
        n = 0
        while n < prob.steps:
            if n % prob.checkpoint == 0:
                ckpts[n] = grid.save_state()
            seg = min(prob.checkpoint - n % prob.checkpoint, prob.steps - n)
            rows.append(_run_forward(grid, adj, seg, first))
            n += seg
        vals = torch.cat(rows).double()                    # (window, n_probes)
        ibar = (vals ** 2).mean(dim=0)
        diff = ibar - prob.target
        tnorm = torch.linalg.norm(prob.target)
        loss = torch.linalg.norm(diff) / tnorm
        ctx.prob, ctx.ckpts, ctx.weights = prob, ckpts, (wa, wp)
        ctx.w_device, ctx.w_dtype = w_amp.device, w_amp.dtype
        ctx.save_for_backward(diff, tnorm.reshape(1), loss.reshape(1))
        return loss

    @staticmethod
    def backward(ctx, g_loss):
        diff, tnorm, loss = ctx.saved_tensors
        prob = ctx.prob
        grid, adj, _ = prob.context()
        _set_weights(grid, prob, *ctx.weights)           # another forward may have run since
        # dL/dIbar, then dL/dE^n = dL/dIbar * 2 E^n / window at the probes
        dl_dI = g_loss * diff / (loss * tnorm * tnorm)
        first = prob.steps - prob.window + 1
        adj.reset(prob.steps)
        starts = sorted(ctx.ckpts)
        for s0 in reversed(starts):
            s1 = min(s0 + prob.checkpoint, prob.steps)
            grid.load_state(ctx.ckpts[s0])
            vals = _run_forward(grid, adj, s1 - s0, first).double()   # E^{s1-nrec+1} .. E^{s1}
            nrec = vals.shape[0]
            if nrec:
                dlde = (2.0 / prob.window) * dl_dI.unsqueeze(0) * vals
                dlde = torch.flip(dlde, dims=[0])           # latest first
                pad = torch.zeros((s1 - s0 - nrec, dlde.shape[1]), dtype=dlde.dtype, device=dlde.device)
                adj.step(s1 - s0, torch.cat([dlde, pad]).to(grid.dtype))
            else:
                adj.step(s1 - s0)
        ga, gp = adj.gradient()
        return ga.to(ctx.w_device, ctx.w_dtype), gp.to(ctx.w_device, ctx.w_dtype), None


def beam_loss(w_amp: torch.Tensor, w_phase: torch.Tensor, prob: BeamProblem) -> torch.Tensor:
    return BeamLoss.apply(w_amp, w_phase, prob)
