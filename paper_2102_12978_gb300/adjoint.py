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
"""
from __future__ import annotations

from dataclasses import dataclass

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


def _run_forward(grid, adj, steps, window, record_from):
    """Step `steps` times; return probe rows for steps whose output index
    (1-based, counted from the grid's step at entry) is >= record_from."""
    rows = []
    n0 = grid.n
    for s in range(steps):
        grid.step(1)
        if n0 + s + 1 >= record_from:
            rows.append(adj.probe_read().clone())
    return rows


class BeamLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w_amp: torch.Tensor, w_phase: torch.Tensor, prob: BeamProblem):
        grid = fdtd.Grid(prob.desc)
        grid.set_source(w_amp=w_amp.detach().double().cpu().numpy(),
                        w_phase=w_phase.detach().double().cpu().numpy(), **prob.source)
        adj = fdtd.Adjoint(grid, prob.component, prob.probes)
        first = prob.steps - prob.window + 1          # window = E^first .. E^steps
        ckpts = {}
        rows = []
        n = 0
        while n < prob.steps:
            if n % prob.checkpoint == 0:
                ckpts[n] = grid.save_state()
            seg = min(prob.checkpoint - n % prob.checkpoint, prob.steps - n)
            rows += _run_forward(grid, adj, seg, prob.window, first)
            n += seg
        vals = torch.stack(rows).double()                  # (window, n_probes)
        ibar = (vals ** 2).mean(dim=0)
        diff = ibar - prob.target
        tnorm = torch.linalg.norm(prob.target)
        loss = torch.linalg.norm(diff) / tnorm
        ctx.grid, ctx.adj, ctx.ckpts, ctx.prob = grid, adj, ckpts, prob
        ctx.w_device, ctx.w_dtype = w_amp.device, w_amp.dtype
        ctx.save_for_backward(diff, tnorm.reshape(1), loss.reshape(1))
        return loss

    @staticmethod
    def backward(ctx, g_loss):
        diff, tnorm, loss = ctx.saved_tensors
        prob, grid, adj = ctx.prob, ctx.grid, ctx.adj
        # dL/dIbar, then dL/dE^n = dL/dIbar * 2 E^n / window at the probes
        dl_dI = g_loss * diff / (loss * tnorm * tnorm)
        first = prob.steps - prob.window + 1
        adj.reset(prob.steps)
        starts = sorted(ctx.ckpts)
        for s0 in reversed(starts):
            s1 = min(s0 + prob.checkpoint, prob.steps)
            grid.load_state(ctx.ckpts[s0])
            rows = _run_forward(grid, adj, s1 - s0, prob.window, first)
            nrec = len(rows)
            if nrec:
                vals = torch.stack(rows).double()          # E^{s1-nrec+1} .. E^{s1}
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
