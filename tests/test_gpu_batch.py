"""Batched stepping of several uneven grids (graph engine with each grid in
its own mode, persistent cell engine): each grid must match its own
sequential run of the same arithmetic bit for bit, and the FP64 oracle
within the parity tolerance.  The batch autotuner leaves every grid's state
as it found it."""
import numpy as np
import pytest

import oracle
from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300 import workloads as W
from tests.cases import oracle_grid, oracle_source, rel_l2
from tests.gpu_cases import gpu_grid, host

pytestmark = pytest.mark.gpu


def _cases():
    return [
        W.small(nx=48, ny=40, nz=16, npml=6, r_center=11.0, m=0, theta_deg=20.0, ramp=1.0),
        W.small(nx=64, ny=64, nz=8, npml=8, r_center=14.0, m=2, theta_deg=30.0, pol="circ+", ramp=1.0),
        W.small(nx=37, ny=45, nz=12, npml=6, r_center=9.0, m=1, theta_deg=10.0, pol="x", ramp=1.0),
        W.small(nx=96, ny=33, nz=5, npml=6, r_center=8.0, m=3, theta_deg=25.0, ramp=1.0),
    ]


@pytest.mark.parametrize("engine", [fdtd.BATCH_CELL, fdtd.BATCH_PERSISTENT_CELL])
@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_batched_equals_sequential_bitwise(precision, engine):
    """130 steps = two replays of the 64-step graph (or two 64-step
    persistent launches) plus a 2-step remainder; each engine against the
    single-grid step of the same arithmetic (tile variant 5)."""
    ws = _cases()
    seq = [gpu_grid(w, precision, tile=(5, 4, 1)) for w in ws]
    bat = [gpu_grid(w, precision) for w in ws]
    b = fdtd.Batch(bat, engine=engine)
    assert b.engine == engine
    assert b.work_items > 0
    nsteps = 130
    for g in seq:
        g.step(nsteps)
    b.step(nsteps)
    b.sync()
    for gs, gb in zip(seq, bat):
        assert gb.n == gs.n == nsteps
        for c in range(6):
            assert np.array_equal(host(gs.field(c)), host(gb.field(c))), c
        assert np.array_equal(host(gs.fluence()), host(gb.fluence()))
    b.close()


def test_graph_engine_grid_modes_bitwise():
    """Each grid in its own mode of the graph engine -- cell passes on
    32 x 8 and 32 x 16 blocks, the two-step kernel on a share of the SMs --
    over two 64-step replays equals the same grid stepped alone with that
    tile (tile variants 5 and 7), bit for bit."""
    ws = _cases()
    modes = [fdtd.BATCH_MODE_TWO_STEP, fdtd.BATCH_MODE_CELL8, fdtd.BATCH_MODE_CELL16, fdtd.BATCH_MODE_TWO_STEP]
    tiles = {fdtd.BATCH_MODE_CELL8: (5, 8, 1), fdtd.BATCH_MODE_CELL16: (5, 16, 1), fdtd.BATCH_MODE_TWO_STEP: (7, 16, 1)}
    seq = [gpu_grid(w, "f32", tile=tiles[m]) for w, m in zip(ws, modes)]
    bat = [gpu_grid(w, "f32") for w in ws]
    b = fdtd.Batch(bat)
    for q, m in enumerate(modes):
        b.set_grid_mode(q, m)
        assert b.grid_mode(q) == m
    for g in seq:
        g.step(128)
    b.step(128)
    b.sync()
    for gs, gb in zip(seq, bat):
        assert gb.n == gs.n == 128
        for c in range(6):
            assert np.array_equal(host(gs.field(c)), host(gb.field(c))), c
        assert np.array_equal(host(gs.fluence()), host(gb.fluence()))
    b.close()


def test_two_step_mode_refused_where_it_cannot_run():
    ws = _cases()[:2]
    b = fdtd.Batch([gpu_grid(w, "f64") for w in ws])
    with pytest.raises(fdtd.FDTDError) as e:
        b.set_grid_mode(0, fdtd.BATCH_MODE_TWO_STEP)
    assert e.value.status == fdtd.FDTD_EINVAL
    with pytest.raises(fdtd.FDTDError) as e:
        b.set_grid_mode(0, 7)
    assert e.value.status == fdtd.FDTD_EINVAL
    with pytest.raises(fdtd.FDTDError) as e:
        b.set_engine(fdtd.BATCH_PERSISTENT)   # the persistent TMA engine is no longer built
    assert e.value.status == fdtd.FDTD_EINVAL
    b.close()


def test_batch_autotune_restores_every_grid():
    """The autotuner steps every grid while it times modes and engines; it
    puts back each grid's fields, fluence, step counter and copy parity, and
    the tuned batch then matches the FP64 oracle within the FP32 bound."""
    ws = _cases()
    bat = [gpu_grid(w, "f32") for w in ws]
    b = fdtd.Batch(bat)
    b.step(5)
    b.sync()
    before = [[g.field(c).clone() for c in range(6)] + [g.fluence().clone()] for g in bat]
    engine, modes = b.autotune(steps=4)
    assert engine in (fdtd.BATCH_CELL, fdtd.BATCH_PERSISTENT_CELL)
    assert all(m in (0, 1, 2, 3) for m in modes)
    for g, ref in zip(bat, before):
        assert g.n == 5
        for c in range(6):
            assert np.array_equal(host(g.field(c)), host(ref[c])), c
        assert np.array_equal(host(g.fluence()), host(ref[6]))
    b.step(128 + 3 - 5)
    b.sync()
    for w, g in zip(ws, bat):
        og, os_ = oracle_grid(w), oracle_source(w)
        st = oracle.State(og)
        oracle.run(og, os_, st, 128 + 3)
        for c, ref in enumerate(st.fields()):
            assert rel_l2(host(g.field(c)), ref) <= 1e-4, (w.name, c)
        assert rel_l2(host(g.fluence()), st.fluence) <= 1e-4
    b.close()


def test_batch_engine_switch_keeps_source_phase():
    """Steps split between the engines (a switch between graph replays and
    remainders) match the single-grid steps within the FP64 parity bound."""
    ws = _cases()[:3]
    seq = [gpu_grid(w, "f64", tile=(5, 4, 1)) for w in ws]
    bat = [gpu_grid(w, "f64") for w in ws]
    b = fdtd.Batch(bat)
    b.step(67)
    b.set_engine(fdtd.BATCH_PERSISTENT_CELL)
    b.step(66)
    b.set_engine(fdtd.BATCH_CELL)
    b.step(5)
    b.sync()
    for g in seq:
        g.step(138)
    for gs, gb in zip(seq, bat):
        for c in range(6):
            assert rel_l2(host(gb.field(c)), host(gs.field(c))) <= 1e-12, c
        assert rel_l2(host(gb.fluence()), host(gs.fluence())) <= 1e-12
    b.close()


@pytest.mark.parametrize("engine", [fdtd.BATCH_CELL, fdtd.BATCH_PERSISTENT_CELL])
def test_batched_matches_oracle_f64(engine):
    ws = _cases()
    grids = [gpu_grid(w, "f64") for w in ws]
    b = fdtd.Batch(grids, engine=engine)
    nsteps = 70
    b.step(nsteps)
    b.sync()
    for w, g in zip(ws, grids):
        og, os_ = oracle_grid(w), oracle_source(w)
        st = oracle.State(og)
        oracle.run(og, os_, st, nsteps)
        for c, ref in enumerate(st.fields()):
            assert rel_l2(host(g.field(c)), ref) <= 1e-11, (w.name, c)
        assert rel_l2(host(g.fluence()), st.fluence) <= 1e-11
    b.close()


def test_batched_grid_cannot_step_alone():
    """While in a batch a grid refuses its own steps and source changes
    (the batch holds copies of its arguments); a batch whose grid was put at
    another copy parity refuses to step; after the batch is destroyed the
    grid steps on its own again."""
    ws = _cases()[:2]
    grids = [gpu_grid(w, "f32") for w in ws]
    b = fdtd.Batch(grids)
    b.step(3)
    for call in (lambda: grids[0].step(1), lambda: grids[0].step_timed(1), lambda: grids[0].autotune(1),
                 lambda: grids[0].set_source(r_center=8.0), lambda: grids[0].clear_source(),
                 lambda: grids[0].set_wall_source(plane=2)):
        with pytest.raises(fdtd.FDTDError) as e:
            call()
        assert e.value.status == fdtd.FDTD_ESTATE
    fresh = gpu_grid(ws[0], "f32")
    grids[0].load_state(fresh.save_state())   # step 0, copy parity 0 -- the batch is at parity 1
    with pytest.raises(fdtd.FDTDError) as e:
        b.step(1)
    assert e.value.status == fdtd.FDTD_ESTATE
    b.close()
    grids[0].step(1)
    grids[0].sync()


def test_batch_of_more_grids_than_one_launch_holds():
    """More grids (19) than the cell engine's concurrent graph branches (16):
    grids share branches round-robin."""
    ws = [W.small(nx=40 + 4 * (q % 3), ny=36, nz=6, npml=6, r_center=8.0, m=q % 3, ramp=1.0) for q in range(19)]
    seq = [gpu_grid(w, "f32", tile=(5, 4, 1)) for w in ws]
    bat = [gpu_grid(w, "f32") for w in ws]
    b = fdtd.Batch(bat)
    b.step(9)
    b.sync()
    for g in seq:
        g.step(9)
    for gs, gb in zip(seq, bat):
        for c in range(6):
            assert np.array_equal(host(gs.field(c)), host(gb.field(c))), c
    b.close()


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_persistent_cell_engine_many_uneven_grids(precision):
    """27 grids of uneven shapes (ragged tiles, nz from 1 to 20): two groups
    of launches (24 grids per cooperative launch, then 3), 70 steps (64 + 6)
    on the persistent cell engine and 6 on the graph cell engine, bit for bit
    against each grid's own variant-5 steps."""
    rng = W.rng(W.SEED + 5)
    ws = []
    for q in range(27):
        nx, ny = int(rng.integers(33, 90)), int(rng.integers(30, 80))
        nz = int(rng.integers(1, 21))
        ws.append(W.small(nx=nx, ny=ny, nz=nz, npml=6, r_center=min(nx, ny) / 2 - 9.0, ramp=1.0,
                          m=int(q % 3), theta_deg=float(10 + 2 * q)))
    seq = [gpu_grid(w, precision, tile=(5, 4, 1)) for w in ws]
    bat = [gpu_grid(w, precision) for w in ws]
    b = fdtd.Batch(bat, engine=fdtd.BATCH_PERSISTENT_CELL)
    assert b.engine == fdtd.BATCH_PERSISTENT_CELL
    b.step(70)
    b.set_engine(fdtd.BATCH_CELL)
    b.step(6)
    b.sync()
    for g in seq:
        g.step(76)
    for gs, gb in zip(seq, bat):
        assert gb.n == gs.n == 76
        for c in range(6):
            assert np.array_equal(host(gs.field(c)), host(gb.field(c))), c
        assert np.array_equal(host(gs.fluence()), host(gb.fluence()))
    b.close()


def test_grid_taller_than_one_launch():
    """A grid of 65540 planes, more than one launch's 65535 CTA rows along
    z: tile variant 5 launches its passes in two chunks of planes.  6 FP64
    steps from a seeded random state against the oracle; the graph cell and
    persistent cell batch engines then repeat them bit for bit."""
    w = W.small(nx=8, ny=8, nz=65540, npml=2, steps=6)
    init = W.random_state((w.nz, w.ny, w.nx), seed=W.SEED + 21)
    init[1][:, :, 0] = 0; init[2][:, :, 0] = 0     # tangential E on the i = 0 wall
    init[0][:, 0, :] = 0; init[2][:, 0, :] = 0     # and on the j = 0 wall

    def fresh():
        g = gpu_grid(w, "f64", source=False, fluence=False)
        for c in range(6):
            g.set_field(c, init[c])
        return g

    g = fresh()
    assert g.tile()[0] == 5
    g.step(w.steps)
    g.sync()
    og = oracle_grid(w)
    st = oracle.State(og, fluence=False)
    for c in range(3):
        st.e[c][...] = init[c]
        st.h[c][...] = init[3 + c]
    oracle.run(og, None, st, w.steps)
    for c, ref in enumerate(st.fields()):
        assert rel_l2(host(g.field(c)), ref) <= 1e-11, c
    for engine in (fdtd.BATCH_CELL, fdtd.BATCH_PERSISTENT_CELL):
        gb = fresh()
        b = fdtd.Batch([gb], engine=engine)
        b.step(w.steps)
        b.sync()
        for c in range(6):
            assert np.array_equal(host(gb.field(c)), host(g.field(c))), (engine, c)
        b.close()
