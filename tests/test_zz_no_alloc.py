"""fdtd_fluence_noalloc: the fluence read-out for callers that cannot
allocate device memory (its staging buffer is a fixed array compiled into the
library).  It must return what fdtd_fluence returns, on consecutive calls,
and refuse grids larger than its fixed staging array.  This file is collected
last so that a failure here cannot stop the rest of the GPU suite."""
import numpy as np
import pytest

from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300 import workloads as W
from tests.cases import rel_l2
from tests.gpu_cases import gpu_grid

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-11, "f32": 1e-4}


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_noalloc_fluence_matches_fluence_on_two_calls(precision):
    w = W.small(nx=48, ny=40, nz=16, npml=6, r_center=11.0, ramp=1.0)
    g = gpu_grid(w, precision)
    shape = (w.nz, w.ny, w.nx)
    for steps in (20, 15):               # two calls in a row, more steps between them
        g.step(steps)
        ref = np.empty(shape)
        fdtd.fdtd_fluence(g.handle, ref.ctypes.data, False, False)
        got = np.full(shape, np.nan)
        fdtd.fdtd_fluence_noalloc(g.handle, got.ctypes.data, False, False)
        assert np.isfinite(got).all()
        assert np.abs(ref).max() > 0
        assert rel_l2(got, ref) <= TOL[precision]


def test_noalloc_fluence_rejects_grids_beyond_its_limit():
    limit = fdtd.fdtd_fluence_noalloc_max_cells()
    nz = limit // (128 * 128) + 1
    w = W.small(nx=128, ny=128, nz=nz, npml=8, r_center=30.0, ramp=1.0)
    g = gpu_grid(w, "f32", source=False)
    out = np.empty(1)
    with pytest.raises(fdtd.FDTDError) as e:
        fdtd.fdtd_fluence_noalloc(g.handle, out.ctypes.data, False, False)
    assert e.value.status == fdtd.FDTD_EINVAL
