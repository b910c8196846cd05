"""The GPU reverse-time adjoint against the oracle's pinned adjoint, and the
end-to-end weight gradient (autograd Function with checkpoint recompute)
against central finite differences of the GPU forward."""
import numpy as np
import pytest
import torch

import oracle
from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300 import workloads as W
from paper_2102_12978_gb300.adjoint import BeamProblem, beam_loss
from tests.cases import oracle_grid, oracle_source, rel_l2
from tests.gpu_cases import gpu_grid, host

pytestmark = pytest.mark.gpu

# components of the adjoint state below this fraction of the state's norm are
# compared against that fraction of the state's norm
ADJ_FLOOR = 1e-2


@pytest.mark.parametrize("precision,tol_f,tol_g", [("f64", 1e-11, 1e-10), ("f32", 1e-4, 1e-3)])
def test_adjoint_matches_oracle(precision, tol_f, tol_g):
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=9.0, steps=30, ramp=0.5, theta_deg=25.0)
    amp, ph = W.random_weights(w.nx, w.ny, seed=3)
    g = gpu_grid(w, precision, w_amp=amp, w_phase=ph)
    g.step(w.steps)
    rng = W.rng(9)
    probes = rng.integers(0, w.nx * w.ny * w.nz, size=64)
    window = 6
    dlde = rng.standard_normal((window, probes.size))
    adj = fdtd.Adjoint(g, fdtd.EY, probes)
    adj.reset(w.steps)
    adj.step(window, torch.tensor(dlde, device=g.device))
    adj.step(w.steps - window)
    assert adj.position == 0
    ga, gp = (host(t) for t in adj.gradient())

    og = oracle_grid(w)
    src = oracle_source(w, w_amp=amp, w_phase=ph)
    ao = oracle.State(og, fluence=False)
    gao = np.zeros((w.ny, w.nx)); gpo = np.zeros((w.ny, w.nx))
    for r, n in enumerate(reversed(range(w.steps))):
        if r < window:
            np.add.at(ao.e[1].reshape(-1), probes, dlde[r])
        oracle.adjoint_step(og, src, ao, n, gao, gpo)
    # per-component relative L2; a component whose norm is below FLOOR of the
    # whole adjoint state's norm is measured against FLOOR x that norm instead
    # (its rounding comes from the larger components it is coupled to)
    refs = ao.fields()
    total = np.sqrt(sum(float(np.sum(r ** 2)) for r in refs))
    errs, rels = [], []
    for c, r in enumerate(refs):
        diff = float(np.linalg.norm(host(adj.field(c)) - r))
        errs.append(diff / max(float(np.linalg.norm(r)), ADJ_FLOOR * total))
        rels.append(rel_l2(host(adj.field(c)), r))
    print("adjoint per-component rel-L2", precision, rels, "norm / state norm",
          [float(np.linalg.norm(r)) / total for r in refs])
    assert max(errs) <= tol_f, (errs, rels)
    assert rel_l2(ga, gao) <= tol_g, rel_l2(ga, gao)
    assert rel_l2(gp, gpo) <= tol_g, rel_l2(gp, gpo)


def _problem(w, precision, steps, window, checkpoint, seed=4, tile=None):
    d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant,
                            precision=precision, fluence=False)
    rng = W.rng(seed)
    # dominant-component probes inside the ring, every plane
    i = np.arange(w.nx)[None, :]
    j = np.arange(w.ny)[:, None]
    r = np.hypot(i - w.nx / 2, j + 0.5 - w.ny / 2)
    r0 = 0.383 / np.sin(w.theta) / w.dx              # central-lobe radius in cells
    cols = np.flatnonzero((r < min(w.r_center - 2, 3 * r0)).ravel())
    probes = (np.arange(w.nz)[:, None] * (w.nx * w.ny) + cols[None, :]).ravel()
    target = torch.tensor(0.5 + rng.random(probes.size), dtype=torch.float64, device="cuda")
    src = dict(m=w.m, theta=w.theta, pol=w.pol, r_center=w.r_center, thickness=w.thickness, ramp=w.ramp)
    return BeamProblem(d, src, fdtd.EY, probes, target, steps, window, checkpoint, tile=tile)


def _fd_check(w, precision, steps, window, checkpoint, n_weights, h, tol, seed=4, tile=None):
    """Adjoint gradient in `precision` against central differences of the
    FP64 forward (one column moves the loss by ~1/n_columns of its value, far
    below FP32 rounding of the forward, so the differences are taken in FP64)."""
    prob = _problem(w, precision, steps, window, checkpoint, seed, tile=tile)
    prob64 = _problem(w, "f64", steps, window, checkpoint, seed)
    amp0, ph0 = W.random_weights(w.nx, w.ny, seed=seed)
    wa = torch.tensor(amp0, requires_grad=True)
    wp = torch.tensor(ph0, requires_grad=True)
    loss = beam_loss(wa, wp, prob)
    loss.backward()
    ga, gp = wa.grad.cpu().numpy(), wp.grad.cpu().numpy()
    # random antenna columns (those with a nonzero gradient)
    rng = W.rng(seed + 1)
    ring = np.flatnonzero(np.abs(ga).ravel() > 0)
    picks = rng.choice(ring, size=n_weights, replace=False)
    worst = 0.0
    for q, col in enumerate(picks):
        jj, ii = divmod(int(col), w.nx)
        which = "amp" if q % 2 == 0 else "phase"
        a1, a2, p1, p2 = amp0.copy(), amp0.copy(), ph0.copy(), ph0.copy()
        if which == "amp":
            a1[jj, ii] += h; a2[jj, ii] -= h
            grad = ga[jj, ii]
        else:
            p1[jj, ii] += h; p2[jj, ii] -= h
            grad = gp[jj, ii]
        lp = beam_loss(torch.tensor(a1), torch.tensor(p1), prob64).item()
        lm = beam_loss(torch.tensor(a2), torch.tensor(p2), prob64).item()
        fd = (lp - lm) / (2 * h)
        scale = max(abs(fd), 1e-3 * np.abs(np.concatenate([ga.ravel(), gp.ravel()])).max())
        worst = max(worst, abs(fd - grad) / scale)
    assert worst <= tol, worst
    return worst


def test_gradient_fd_small_f64():
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=10.0, ramp=0.5, theta_deg=25.0)
    _fd_check(w, "f64", steps=60, window=12, checkpoint=25, n_weights=8, h=1e-6, tol=1e-6)


def test_gradient_fd_small_f32():
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=10.0, ramp=0.5, theta_deg=25.0)
    _fd_check(w, "f32", steps=60, window=12, checkpoint=25, n_weights=8, h=1e-5, tol=1e-3)


def test_gradient_fd_adjoint_workload_f32():
    """The 384x384x96 (lambda/20, theta = 15 deg, 3-cell ring at 0.8 of the
    interior half-width) workload over its full 5000 steps in FP32 (the
    steps before the loss window on the two-step kernel), checkpoints every
    250 steps, the loss on the last 250 steps: 20 random weights against
    central differences of the FP64 forward, <= 1e-3 relative."""
    w = W.config5()
    assert w.steps == 5000
    worst = _fd_check(w, "f32", steps=5000, window=250, checkpoint=250, n_weights=20, h=1e-5, tol=1e-3,
                      tile=(7, 16, 1))
    print("config 5, 5000 steps: worst relative gradient error", worst)


def test_forward_reuses_one_grid():
    """Every forward of a problem runs on the same grid, restarted from its
    zeroed initial state: a loss evaluated twice, with other weights in
    between, is the same to the last bit, and its gradient too."""
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=10.0, ramp=0.5, theta_deg=25.0)
    prob = _problem(w, "f32", steps=40, window=10, checkpoint=16)
    amp0, ph0 = W.random_weights(w.nx, w.ny, seed=8)
    wa = torch.tensor(amp0, requires_grad=True)
    wp = torch.tensor(ph0, requires_grad=True)
    l1 = beam_loss(wa, wp, prob)
    grid = prob.context()[0]
    beam_loss(torch.tensor(amp0 * 1.1), torch.tensor(ph0 + 0.2), prob)
    l1.backward()
    g1 = (wa.grad.clone(), wp.grad.clone())
    wa.grad = None
    wp.grad = None
    l2 = beam_loss(wa, wp, prob)
    l2.backward()
    assert prob.context()[0] is grid
    assert l1.item() == l2.item()
    assert torch.equal(g1[0], wa.grad) and torch.equal(g1[1], wp.grad)
