"""Element-by-element parity of the CUDA path (through the C ABI) with the
FP64 oracle on the same seeded inputs.

Tolerances (relative L2 per field component and for the fluence):
  FP64 GPU vs oracle  <= 1e-11
  FP32 GPU vs oracle  <= 1e-4
The integer decisions (which Yee points belong to the antenna) are compared
exactly through the point counts.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2102_12978_gb300 import workloads as W
from tests.cases import oracle_grid, oracle_source, rel_l2
from tests.gpu_cases import gpu_grid, host

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-11, "f32": 1e-4}


def _compare(w, precision, tile=None, npml=None, source=True, init=None, fluence=True):
    og = oracle_grid(w, npml=npml)
    os_ = oracle_source(w) if source else None
    st = oracle.State(og, fluence=fluence)
    g = gpu_grid(w, precision, npml=npml, source=source, tile=tile, fluence=fluence)
    assert abs(g.dt - og.dt) <= 1e-15 * og.dt
    if init is not None:
        for c in range(3):
            st.e[c][...] = init[c]
            st.h[c][...] = init[3 + c]
        for c in range(6):
            g.set_field(c, init[c])
    oracle.run(og, os_, st, w.steps)
    g.step(w.steps)
    g.sync()
    errs = {}
    for c, ref in enumerate(st.fields()):
        got = host(g.field(c))
        assert np.isfinite(got).all(), "non-finite field values"
        errs["ExEyEzHxHyHz"[2 * c:2 * c + 2]] = rel_l2(got, ref)
    if fluence:
        got = host(g.fluence())
        assert np.isfinite(got).all(), "non-finite fluence values"
        errs["fluence"] = rel_l2(got, st.fluence)
    if source:
        counts = oracle.antenna_counts(og, os_)
        assert [g.antenna_points(c) for c in range(6)] == counts
    return errs


def _assert(errs, precision):
    bad = {k: v for k, v in errs.items() if not (v <= TOL[precision])}
    assert not bad, (precision, errs)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(48, 40, 16), (45, 37, 11), (64, 32, 5)])
def test_small_grids_match_oracle(precision, shape):
    nx, ny, nz = shape
    w = W.small(nx=nx, ny=ny, nz=nz, npml=6, r_center=min(nx, ny) / 2 - 8.5, steps=60, ramp=1.0)
    _assert(_compare(w, precision), precision)


TILES = [(1, 4, 1), (1, 8, 3), (1, 8, 64), (2, 4, 1), (2, 8, 3), (2, 8, 64), (3, 4, 1), (3, 8, 3), (3, 16, 16),
         (3, 8, 64), (4, 4, 1), (4, 8, 3), (4, 16, 16), (4, 8, 64), (5, 4, 1), (5, 8, 1), (5, 16, 1), (6, 4, 1), (6, 8, 1), (6, 16, 1), (0, 4, 1), (0, 8, 3), (0, 16, 16), (0, 8, 64)]


def _skip_missing(tile, precision):
    """The TMA variants (1, 2, 4) have no FP64 32x16 tile."""
    if precision == "f64" and tile[1] == 16 and tile[0] in (1, 2, 4):
        pytest.skip("no FP64 32x16 TMA tile")


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_tilings_and_z_segments_agree(tile, precision):
    """Every (variant, ty, lz) tiling -- TMA-staged and plain-load kernels,
    one-pass and two-pass steps, one-plane z segments, ragged tiles --
    matches the oracle."""
    _skip_missing(tile, precision)
    w = W.small(nx=40, ny=36, nz=16, npml=6, r_center=9.0, steps=30, ramp=1.0)
    _assert(_compare(w, precision, tile=tile), precision)


@pytest.mark.parametrize("variant", [1, 2])
def test_tma_f32_tall_tile(variant):
    w = W.small(nx=72, ny=50, nz=12, npml=6, r_center=12.0, steps=30, ramp=1.0)
    _assert(_compare(w, "f32", tile=(variant, 16, 5)), "f32")


@pytest.mark.parametrize("tile", [(1, 8, 5), (1, 4, 12), (2, 8, 5), (2, 4, 3), (2, 16, 12), (3, 8, 5), (3, 4, 12),
                                  (3, 16, 3), (4, 8, 5), (4, 4, 12), (4, 16, 3), (5, 4, 1), (5, 8, 1), (5, 16, 1),
                                  (6, 4, 1), (6, 8, 1), (6, 16, 1)])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_interior_block_classes(tile, precision):
    """A grid wide enough that the kernels meet all three block classes:
    blocks touching the CPML shell, a wall or a ragged edge (every check
    compiled in), interior blocks holding antenna cells, and plain interior
    blocks (no CPML, wall or source code)."""
    _skip_missing(tile, precision)
    w = W.small(nx=136, ny=120, nz=12, npml=6, r_center=30.0, thickness=2.0, steps=40, ramp=1.0)
    _assert(_compare(w, precision, tile=tile), precision)


@pytest.mark.parametrize("kw", [
    dict(m=2, pol="circ+"), dict(m=3, pol="x", mode="TM"), dict(m=1, pol="circ-", inject="tangential"),
    dict(envelope="gauss", T=0.75, T0=1.5), dict(thickness=3.0, r_center=8.0, theta_deg=30.0),
    dict(m=0, pol="z"), dict(m=0, pol="z", mode="TM"), dict(m=1, pol="z", mode="TM", inject="tangential"),
])
def test_source_variants_match_oracle(kw):
    base = dict(nx=44, ny=40, nz=12, npml=6, r_center=9.0, steps=50, ramp=1.0)
    base.update(kw)
    w = W.small(**base)
    _assert(_compare(w, "f64"), "f64")


@pytest.mark.parametrize("tile", [(1, 8, 5), (3, 8, 5), (4, 8, 5), (5, 8, 1), (6, 8, 1)])
def test_without_fluence_accumulator(tile):
    """Grids created without a fluence accumulator step the fields alone."""
    w = W.small(nx=44, ny=40, nz=12, npml=6, r_center=9.0, steps=40, ramp=1.0)
    _assert(_compare(w, "f32", tile=tile, fluence=False), "f32")


def test_source_free_pec_random_state():
    """npml = 0 (PEC box), no antenna, seeded random state: the bare Yee update."""
    w = W.small(nx=33, ny=20, nz=7, npml=0, steps=40)
    init = W.random_state((w.nz, w.ny, w.nx))
    init[1][:, :, 0] = 0; init[2][:, :, 0] = 0
    init[0][:, 0, :] = 0; init[2][:, 0, :] = 0
    _assert(_compare(w, "f64", npml=0, source=False, init=init), "f64")


@pytest.mark.parametrize("tile", [None, (3, 8, 1), (4, 8, 1), (4, 4, 2), (5, 8, 1), (6, 8, 1)])
def test_nz_one_and_two(tile):
    for nz in (1, 2):
        w = W.small(nx=40, ny=40, nz=nz, npml=6, r_center=9.0, steps=25, ramp=1.0)
        _assert(_compare(w, "f64", tile=tile), "f64")


def test_config1_full_parity_f64():
    """64x64x32, dx = lambda/16, theta = 20 deg, x-polarised, tangential
    injection on a 1-cell ring of radius 12, 8-cell CPML, 400 steps: every
    field and the fluence against the oracle."""
    w = W.config1()
    errs = _compare(w, "f64")
    print("config1 f64 rel-L2:", errs)
    _assert(errs, "f64")


def test_config1_full_parity_f32():
    w = W.config1()
    errs = _compare(w, "f32")
    print("config1 f32 rel-L2:", errs)
    _assert(errs, "f32")


def test_state_save_load_roundtrip():
    """Checkpoint / resume: run 20, save, run 20, load, run 20 == run 40."""
    import torch
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=9.0, steps=20, ramp=1.0)
    g = gpu_grid(w, "f64")
    g.step(20)
    buf = g.save_state()
    g.step(20)
    a = [host(g.field(c)) for c in range(6)] + [host(g.fluence())]
    g.load_state(buf)
    assert g.n == 20
    g.step(20)
    b = [host(g.field(c)) for c in range(6)] + [host(g.fluence())]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_fluence_reset_window():
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=9.0, steps=20, ramp=1.0)
    g = gpu_grid(w, "f64")
    g.step(10)
    f1 = host(g.fluence(reset=True))
    g.step(10)
    f2 = host(g.fluence())
    og, os_ = oracle_grid(w), oracle_source(w)
    st = oracle.State(og)
    oracle.run(og, os_, st, 10)
    assert rel_l2(f1, st.fluence) < 1e-11
    st.fluence[...] = 0
    oracle.run(og, os_, st, 10)
    assert rel_l2(f2, st.fluence) < 1e-11


@pytest.mark.parametrize("tile,npass", [((1, 8, 8), 1), ((3, 4, 8), 2), ((4, 8, 8), 2), ((5, 4, 1), 2),
                                        ((6, 4, 1), 1)])
def test_step_timed_steps_like_step(tile, npass):
    """fdtd_step_timed advances the grid exactly like fdtd_step and reports
    one duration per kernel of a step."""
    w = W.small(nx=48, ny=40, nz=16, npml=6, r_center=10.0, steps=12, ramp=1.0)
    a = gpu_grid(w, "f32", tile=tile)
    b = gpu_grid(w, "f32", tile=tile)
    a.step(w.steps)
    ms = b.step_timed(w.steps)
    assert len(ms) == npass and all(t > 0 for t in ms)
    assert a.n == b.n == w.steps
    for c in range(6):
        assert np.array_equal(host(a.field(c)), host(b.field(c)))
    assert np.array_equal(host(a.fluence()), host(b.fluence()))
