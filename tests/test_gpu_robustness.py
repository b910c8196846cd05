"""Edge cases of the GPU path: grids smaller than one tile (every variant,
every cell against the oracle), and the bounded device wait: a withheld bulk
copy (host-side fault injection) makes the wait expire, the host reads
FDTD_ETIMEOUT, and the device stays usable."""
import numpy as np
import pytest

from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300 import workloads as W
from tests.test_gpu_parity import _assert, _compare

pytestmark = pytest.mark.gpu

VARIANTS = [(0, 4, 1), (1, 4, 1), (1, 8, 2), (2, 8, 2), (3, 4, 1), (4, 4, 1), (5, 4, 1), (5, 16, 1), (6, 4, 1)]


def _random_pec_state(w):
    init = W.random_state((w.nz, w.ny, w.nx), seed=11)
    init[1][:, :, 0] = 0; init[2][:, :, 0] = 0     # tangential E on the i = 0 wall
    init[0][:, 0, :] = 0; init[2][:, 0, :] = 0     # and on the j = 0 wall
    return init


@pytest.mark.parametrize("tile", VARIANTS)
@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shape,npml", [((13, 7, 5), 1), ((8, 8, 8), 2), ((4, 4, 4), 0), ((33, 9, 3), 2)])
def test_grids_smaller_than_a_tile(shape, npml, precision, tile):
    nx, ny, nz = shape
    w = W.small(nx=nx, ny=ny, nz=nz, npml=npml, steps=12)
    _assert(_compare(w, precision, tile=tile, npml=npml, source=False, init=_random_pec_state(w)), precision)


@pytest.mark.parametrize("tile", VARIANTS)
def test_tiny_grid_with_antenna(tile):
    w = W.small(nx=13, ny=11, nz=5, npml=1, r_center=1.5, thickness=1.0, steps=20, ramp=0.2)
    _assert(_compare(w, "f64", tile=tile, npml=1), "f64")


def test_expired_device_wait_reports_timeout():
    w = W.small(nx=48, ny=40, nz=16, npml=6, r_center=11.0, steps=6, ramp=1.0)
    d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, precision="f32")
    g = fdtd.Grid(d)
    g.set_source(m=w.m, theta=w.theta, pol=w.pol, r_center=w.r_center, thickness=w.thickness, ramp=w.ramp)
    g.set_tile(1, 8, 8)
    g.step(2)
    g.sync()
    g.inject_fault(1)
    g.step(1)
    with pytest.raises(fdtd.FDTDError) as e:
        g.sync()
    assert e.value.status == fdtd.FDTD_ETIMEOUT
    g.sync()                      # the error word was cleared with the report
    g.step(2)                     # the fault applied to one step only
    g.sync()
    g.close()
    # the device context is still usable: a fresh grid matches the oracle
    _assert(_compare(W.small(nx=40, ny=36, nz=8, npml=6, r_center=9.0, steps=20, ramp=1.0), "f32",
                     tile=(1, 8, 8)), "f32")


def test_fault_hook_rejects_unknown_kinds():
    w = W.small(nx=16, ny=16, nz=4, npml=2)
    g = fdtd.Grid(fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz))
    with pytest.raises(fdtd.FDTDError) as e:
        g.inject_fault(7)
    assert e.value.status == fdtd.FDTD_EINVAL
    g.close()


def test_expired_grid_barrier_reports_timeout():
    """The persistent cell engine's grid barrier: a lost CTA (host-side fault
    hook) makes the other CTAs' bounded waits expire; the host reads
    FDTD_ETIMEOUT, the barrier and error word are reset, and the batch then
    steps correctly (bit for bit against fresh single grids from the same
    saved state)."""
    from tests.gpu_cases import gpu_grid, host
    ws = [W.small(nx=48, ny=40, nz=8, npml=6, r_center=11.0, ramp=1.0),
          W.small(nx=37, ny=45, nz=6, npml=6, r_center=9.0, m=1, ramp=1.0)]
    bat = [gpu_grid(w, "f32") for w in ws]
    b = fdtd.Batch(bat, engine=fdtd.BATCH_PERSISTENT_CELL)
    b.step(4)
    b.sync()
    b.inject_fault(1)
    b.step(2)
    with pytest.raises(fdtd.FDTDError) as e:
        b.sync()
    assert e.value.status == fdtd.FDTD_ETIMEOUT
    b.sync()                      # cleared with the report
    # restart every grid from a known state and compare with single grids
    seq = [gpu_grid(w, "f32", tile=(5, 4, 1)) for w in ws]
    for gs, gb in zip(seq, bat):
        gb.load_state(gs.save_state())
    b.step(10)
    b.sync()
    for g in seq:
        g.step(10)
    for gs, gb in zip(seq, bat):
        for c in range(6):
            assert np.array_equal(host(gs.field(c)), host(gb.field(c))), c
    b.close()
    with pytest.raises(fdtd.FDTDError) as e:
        fdtd.Batch([gpu_grid(ws[0], "f32")]).inject_fault(5)
    assert e.value.status == fdtd.FDTD_EINVAL


def test_entry_points_refuse_a_grid_of_another_device():
    """A grid belongs to the device current at its creation: with another
    device current, every call that would queue work for it or touch its
    memory returns EINVAL and queues nothing (the step counter and the
    fields stay as they were)."""
    import torch
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=9.0, steps=4, ramp=1.0)
    d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant, precision="f32")
    g = fdtd.Grid(d)
    g.set_source(m=w.m, theta=w.theta, r_center=w.r_center, thickness=w.thickness, ramp=w.ramp)
    g.step(3)
    before = g.field(fdtd.EY).clone()
    dev = torch.cuda.current_device()
    g.debug_set_device(dev + 1)
    shape = (w.nz, w.ny, w.nx)
    out = np.zeros(shape)
    calls = {
        "step": lambda: g.step(1),
        "fluence": lambda: fdtd.fdtd_fluence(g.handle, out.ctypes.data, False, False),
        "get_field": lambda: fdtd.fdtd_get_field(g.handle, fdtd.EY, out.ctypes.data, False),
        "set_source": lambda: g.set_source(m=w.m, theta=w.theta, r_center=w.r_center, thickness=w.thickness),
        "sync": lambda: g.sync(),
    }
    for name, call in calls.items():
        with pytest.raises(fdtd.FDTDError) as e:
            call()
        assert e.value.status == fdtd.FDTD_EINVAL, name
    g.debug_set_device(dev)
    assert g.n == 3
    assert torch.equal(g.field(fdtd.EY), before)
