"""Tile variant 7: two Yee steps per launch (temporal blocking), FP32.

Element-by-element parity with the FP64 oracle (relative L2 <= 1e-4 per
field component and for the fluence) on grids that span several overlapping
windows with ragged last windows in x and y, odd step counts (the last step
runs as one cell-pass step), thin and one-plane z extents, grids smaller than
one window, every source variant, random states with every CPML shell busy,
and the full-size 256 x 256 x 128 workload in the launch configuration the
bench times.  Also: checkpoint / resume and switching tile variants between
launches (the E-side psi changes copy with every launch of variant 7), and
agreement with the cell passes (variant 5), which evaluate the same
arithmetic one step at a time."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300 import workloads as W
from tests.cases import oracle_grid, oracle_source, rel_l2
from tests.gpu_cases import gpu_grid, host
from tests.test_gpu_parity import _assert, _compare

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("ty", [16, 8])
@pytest.mark.parametrize("shape,steps", [((48, 40, 16), 60), ((45, 37, 11), 61), ((64, 32, 5), 40),
                                         ((100, 90, 7), 31), ((61, 75, 3), 20)])
def test_windows_and_ragged_edges_match_oracle(shape, steps, ty):
    nx, ny, nz = shape
    w = W.small(nx=nx, ny=ny, nz=nz, npml=6, r_center=min(nx, ny) / 2 - 8.5, steps=steps, ramp=1.0)
    _assert(_compare(w, "f32", tile=(7, ty, 1)), "f32")


@pytest.mark.parametrize("nz", [1, 2, 3])
def test_thin_z_extents(nz):
    w = W.small(nx=40, ny=36, nz=nz, npml=6, r_center=9.0, steps=24, ramp=1.0)
    _assert(_compare(w, "f32", tile=(7, 16, 1)), "f32")


def _random_pec_state(w, seed=17):
    init = W.random_state((w.nz, w.ny, w.nx), seed=seed)
    init[1][:, :, 0] = 0; init[2][:, :, 0] = 0     # tangential E on the i = 0 wall
    init[0][:, 0, :] = 0; init[2][:, 0, :] = 0     # and on the j = 0 wall
    return init


@pytest.mark.parametrize("ty", [16, 8])
@pytest.mark.parametrize("shape,npml", [((13, 7, 5), 1), ((8, 8, 8), 2), ((4, 4, 4), 0), ((33, 9, 3), 2),
                                        ((70, 44, 6), 8), ((29, 30, 4), 0)])
def test_random_states_every_shell_busy(shape, npml, ty):
    """A random state in every cell: the CPML shells, the walls and the
    window overlaps all carry values from the first step."""
    nx, ny, nz = shape
    w = W.small(nx=nx, ny=ny, nz=nz, npml=npml, steps=14)
    _assert(_compare(w, "f32", tile=(7, ty, 1), npml=npml, source=False, init=_random_pec_state(w)), "f32")


@pytest.mark.parametrize("kw", [
    dict(m=2, pol="circ+"), dict(m=3, pol="x", mode="TM"), dict(m=1, pol="circ-", inject="tangential"),
    dict(envelope="gauss", T=0.75, T0=1.5), dict(thickness=3.0, r_center=8.0, theta_deg=30.0),
    dict(m=0, pol="z"), dict(m=1, pol="z", mode="TM", inject="tangential"),
])
def test_source_variants_match_oracle(kw):
    base = dict(nx=44, ny=40, nz=12, npml=6, r_center=9.0, steps=50, ramp=1.0)
    base.update(kw)
    w = W.small(**base)
    _assert(_compare(w, "f32", tile=(7, 16, 1)), "f32")


def test_without_fluence():
    w = W.small(nx=52, ny=41, nz=9, npml=6, r_center=10.0, steps=30, ramp=1.0)
    _assert(_compare(w, "f32", tile=(7, 16, 1), fluence=False), "f32")


def test_interior_windows_with_antenna():
    """Windows far from every wall, some holding antenna columns."""
    w = W.small(nx=136, ny=120, nz=12, npml=6, r_center=30.0, thickness=2.0, steps=40, ramp=1.0)
    _assert(_compare(w, "f32", tile=(7, 16, 1)), "f32")


def test_matches_cell_passes():
    """Variant 7 evaluates each step with the arithmetic of the cell passes
    (variant 5) in the same order; the two agree far inside the FP32
    tolerance after 60 steps."""
    w = W.small(nx=72, ny=66, nz=10, npml=6, r_center=16.0, steps=60, ramp=1.0)
    a = gpu_grid(w, "f32", tile=(7, 16, 1))
    b = gpu_grid(w, "f32", tile=(5, 4, 1))
    a.step(w.steps)
    b.step(w.steps)
    worst = 0.0
    for c in range(6):
        worst = max(worst, rel_l2(host(a.field(c)), host(b.field(c))))
    worst = max(worst, rel_l2(host(a.fluence()), host(b.fluence())))
    print("variant 7 vs variant 5, worst rel-L2:", worst)
    assert worst <= 1e-6, worst


def test_switching_variants_and_checkpoints():
    """Runs that mix variant 7 with single-step variants (the E-side psi
    changes copy with every launch of variant 7), saved and restored in the
    middle, match one oracle run."""
    w = W.small(nx=50, ny=46, nz=8, npml=6, r_center=11.0, steps=45, ramp=1.0)
    og, os_ = oracle_grid(w), oracle_source(w)
    st = oracle.State(og)
    oracle.run(og, os_, st, w.steps)
    g = gpu_grid(w, "f32", tile=(7, 16, 1))
    g.step(7)                        # 3 launches of variant 7 and one cell-pass step
    g.set_tile(3, 8, 3)
    g.step(4)
    g.set_tile(7, 8, 1)
    g.step(10)
    saved = g.save_state()
    n_saved = g.n
    g.set_tile(5, 4, 1)
    g.step(5)                        # diverge, then restore
    g.load_state(saved)
    assert g.n == n_saved
    g.set_tile(7, 16, 1)
    g.step(w.steps - n_saved)
    g.sync()
    errs = {c: rel_l2(host(g.field(c)), ref) for c, ref in enumerate(st.fields())}
    errs["fluence"] = rel_l2(host(g.fluence()), st.fluence)
    _assert(errs, "f32")


def test_timed_steps_match_plain_steps():
    """fdtd_step_timed (CUDA events around every launch) runs the same
    arithmetic as fdtd_step."""
    w = W.small(nx=48, ny=40, nz=8, npml=6, r_center=11.0, steps=20, ramp=1.0)
    a = gpu_grid(w, "f32", tile=(7, 16, 1))
    b = gpu_grid(w, "f32", tile=(7, 16, 1))
    a.step(w.steps)
    ms = b.step_timed(w.steps)
    assert len(ms) == 1 and ms[0] > 0
    for c in range(6):
        assert torch.equal(a.field(c), b.field(c))
    assert torch.equal(a.fluence(), b.fluence())


def test_config2_full_size():
    """256 x 256 x 128, the bench workload, in the configuration the bench
    times (variant 7, 32 x 16 windows), 40 steps against the oracle."""
    w = dataclasses.replace(W.config2(), steps=40)
    errs = _compare(w, "f32", tile=(7, 16, 1))
    print(w.name, "variant 7", {k: f"{v:.2e}" for k, v in errs.items()})
    _assert(errs, "f32")


def test_work_split_weights_change_no_result():
    """The CTAs' work ranges (fdtd_set_balance) decide only which CTA
    computes which planes of a window: the results are bit for bit equal."""
    w = W.small(nx=100, ny=90, nz=9, npml=8, r_center=20.0, steps=12, ramp=1.0)
    runs = []
    for ws, wa in ((0.0, 0.0), (2.0, 5.0), (0.25, 0.2)):
        g = gpu_grid(w, "f32", tile=(7, 16, 1))
        g.set_balance(ws, wa)
        assert g.balance() == pytest.approx((ws, wa))
        g.step(w.steps)
        runs.append([g.field(c) for c in range(6)] + [g.fluence()])
    for other in runs[1:]:
        for x, y in zip(runs[0], other):
            assert torch.equal(x, y)


@pytest.mark.parametrize("ty", [16, 8])
def test_measured_balance_changes_no_result(ty):
    """fdtd_measure_balance runs one measuring launch on a saved copy of the
    state (the grid's state and step count are restored), then balances the
    ranges on the measured per-window costs: the results are bit for bit
    those of the weight-balanced ranges, and fdtd_set_balance returns to the
    weights."""
    w = W.small(nx=100, ny=90, nz=9, npml=8, r_center=20.0, steps=12, ramp=1.0)
    a = gpu_grid(w, "f32", tile=(7, ty, 1))
    b = gpu_grid(w, "f32", tile=(7, ty, 1))
    a.step(4)
    b.step(4)
    n = b.n
    before = [b.field(c).clone() for c in range(6)] + [b.fluence().clone()]
    b.measure_balance()
    assert b.balance() == (-1.0, -1.0) and b.n == n
    for x, y in zip(before, [b.field(c) for c in range(6)] + [b.fluence()]):
        assert torch.equal(x, y)
    a.step(w.steps - 4)
    b.step(w.steps - 4)
    for c in range(6):
        assert torch.equal(a.field(c), b.field(c))
    assert torch.equal(a.fluence(), b.fluence())
    b.set_balance(0.3, 0.2)
    assert b.balance() == pytest.approx((0.3, 0.2))


def test_measured_balance_needs_variant_7():
    w = W.small(nx=48, ny=40, nz=8, npml=6, r_center=11.0, steps=4, ramp=1.0)
    g = gpu_grid(w, "f32", tile=(5, 4, 1))
    with pytest.raises(fdtd.FDTDError) as e:
        g.measure_balance()
    assert e.value.status == fdtd.FDTD_EINVAL


@pytest.mark.parametrize("ty", [16, 8])
@pytest.mark.parametrize("shape", [(100, 90, 9), (200, 150, 12), (61, 75, 3)])
def test_interleaved_window_order_changes_no_result(shape, ty):
    """lz = 2 interleaves the window rows in the CTAs' work (x-neighbours
    march side by side); which CTA computes which window changes, the
    results do not, with the weight-balanced and the refined ranges."""
    nx, ny, nz = shape
    w = W.small(nx=nx, ny=ny, nz=nz, npml=6, r_center=min(nx, ny) / 2 - 8.5, steps=14, ramp=1.0)
    a = gpu_grid(w, "f32", tile=(7, ty, 1))
    b = gpu_grid(w, "f32", tile=(7, ty, 2))
    c = gpu_grid(w, "f32", tile=(7, ty, 2))
    c.measure_balance()
    for g in (a, b, c):
        g.step(w.steps)
    for g in (b, c):
        for comp in range(6):
            assert torch.equal(a.field(comp), g.field(comp))
        assert torch.equal(a.fluence(), g.fluence())
