"""fdtd_fluence_noalloc: the fluence read-out for callers that cannot
allocate device memory (its staging buffer is a fixed array compiled into the
library).  It must return exactly what fdtd_fluence returns (both run the same
export kernel on the same accumulator, so the results are bit for bit equal),
on consecutive calls, to host and to device destinations, reset the
accumulator as fdtd_fluence does, and refuse grids larger than its fixed
staging array or a grid whose device is not current.  This file is collected
last so that a failure here cannot stop the rest of the GPU suite."""
import numpy as np
import pytest
import torch

from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300 import workloads as W
from tests.gpu_cases import gpu_grid

pytestmark = pytest.mark.gpu


def _read(fn, g, shape, on_device, reset=False):
    if on_device:
        out = torch.full(shape, float("nan"), dtype=torch.float64, device=g.device)
        fn(g.handle, out.data_ptr(), True, reset)
        return out.cpu().numpy()
    out = np.full(shape, np.nan)
    fn(g.handle, out.ctypes.data, False, reset)
    return out


@pytest.mark.parametrize("on_device", [False, True])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_fluence_matches_fluence_on_two_calls(precision, on_device):
    w = W.small(nx=48, ny=40, nz=16, npml=6, r_center=11.0, ramp=1.0)
    g = gpu_grid(w, precision)
    shape = (w.nz, w.ny, w.nx)
    for steps in (20, 15):               # two calls in a row, more steps between them
        g.step(steps)
        ref = _read(fdtd.fdtd_fluence, g, shape, on_device)
        got = _read(fdtd.fdtd_fluence_noalloc, g, shape, on_device)
        assert np.isfinite(got).all()
        assert np.abs(ref).max() > 0
        assert np.array_equal(got, ref)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_reset_matches_fluence_reset(precision):
    """reset = 1 returns the accumulated fluence and zeroes the accumulator:
    a read-out with no step in between gives zeros, and after more steps both
    read-outs agree with a grid reset by fdtd_fluence."""
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=9.0, ramp=1.0)
    a, b = gpu_grid(w, precision), gpu_grid(w, precision)
    shape = (w.nz, w.ny, w.nx)
    a.step(12)
    b.step(12)
    got = _read(fdtd.fdtd_fluence_noalloc, a, shape, False, reset=True)
    ref = _read(fdtd.fdtd_fluence, b, shape, False, reset=True)
    assert np.abs(ref).max() > 0 and np.array_equal(got, ref)
    assert not _read(fdtd.fdtd_fluence_noalloc, a, shape, True).any()
    assert not _read(fdtd.fdtd_fluence, b, shape, True).any()
    a.step(7)
    b.step(7)
    got = _read(fdtd.fdtd_fluence_noalloc, a, shape, True)
    ref = _read(fdtd.fdtd_fluence, b, shape, True)
    assert np.abs(ref).max() > 0 and np.array_equal(got, ref)


def test_noalloc_fluence_rejects_grids_beyond_its_limit():
    limit = fdtd.fdtd_fluence_noalloc_max_cells()
    nz = limit // (128 * 128) + 1
    w = W.small(nx=128, ny=128, nz=nz, npml=8, r_center=30.0, ramp=1.0)
    g = gpu_grid(w, "f32", source=False)
    out = np.empty(1)
    with pytest.raises(fdtd.FDTDError) as e:
        fdtd.fdtd_fluence_noalloc(g.handle, out.ctypes.data, False, False)
    assert e.value.status == fdtd.FDTD_EINVAL


def test_noalloc_fluence_refuses_a_grid_of_another_device():
    w = W.small(nx=40, ny=36, nz=8, npml=6, r_center=9.0, ramp=1.0)
    g = gpu_grid(w, "f32")
    g.step(5)
    shape = (w.nz, w.ny, w.nx)
    ref = _read(fdtd.fdtd_fluence, g, shape, False)
    g.debug_set_device(torch.cuda.current_device() + 1)
    out = np.full(shape, np.nan)
    with pytest.raises(fdtd.FDTDError) as e:
        fdtd.fdtd_fluence_noalloc(g.handle, out.ctypes.data, False, False)
    assert e.value.status == fdtd.FDTD_EINVAL
    assert np.isnan(out).all()           # nothing was queued
    g.debug_set_device(torch.cuda.current_device())
    assert np.array_equal(_read(fdtd.fdtd_fluence_noalloc, g, shape, False), ref)
