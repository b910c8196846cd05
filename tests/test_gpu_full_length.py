"""FP32 error at the full run lengths of the benchmark configurations.

The FP64 GPU path matches the oracle to 1e-11 (the parity tests); here it is
the transfer standard over whole runs, where the oracle would take hours: the
FP32 fields and fluence after the full 4000 steps of the 256 x 256 x 128
workload (in the bench's launch configuration and in the cell passes), one
512 x 512 x 64 grid after 6000 steps and one grid of the batched sweep after
3000 steps must stay within 1e-4 relative L2 per field component and for the
fluence.  Large step counts are where the phase arguments omega t of the
source matter (Eq. 12-13): they are evaluated in FP64 on the host.  The
oracle itself referees the first 600 steps of the 256 x 256 x 128 workload,
FP64 and FP32."""
import dataclasses

import numpy as np
import pytest
import torch

import oracle
from paper_2102_12978_gb300 import workloads as W
from tests.cases import oracle_grid, oracle_source, rel_l2
from tests.gpu_cases import gpu_grid, host

pytestmark = pytest.mark.gpu

TOL32 = 1e-4
NAMES = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")


def _rel(x, y) -> float:
    x = x.double(); y = y.double()
    den = float(torch.linalg.vector_norm(y))
    return float(torch.linalg.vector_norm(x - y)) / den


def _f32_against_f64(w, tile):
    a = gpu_grid(w, "f32", tile=tile)
    b = gpu_grid(w, "f64")
    a.step(w.steps)
    b.step(w.steps)
    errs = {n: _rel(a.field(c), b.field(c)) for c, n in enumerate(NAMES)}
    errs["fluence"] = _rel(a.fluence(), b.fluence())
    for t in (*(a.field(c) for c in range(6)), a.fluence()):
        assert torch.isfinite(t).all()
    a.close()
    b.close()
    return errs


@pytest.mark.parametrize("tile", [(7, 16, 1), (5, 4, 1)])
def test_config2_full_run_f32(tile):
    """256 x 256 x 128, all 4000 steps."""
    w = W.config2()
    assert w.steps == 4000
    errs = _f32_against_f64(w, tile)
    print(w.name, tile, {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) <= TOL32, errs


def test_config3_full_run_f32():
    """512 x 512 x 64, l = 3, theta = 30 deg, all 6000 steps."""
    w = W.config3()[5]
    assert (w.m, w.theta_deg, w.steps) == (3, 30.0, 6000)
    errs = _f32_against_f64(w, (7, 16, 1))
    print(w.name, {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) <= TOL32, errs


def test_config4_grid_full_run_f32():
    """The largest grid of the batched sweep (640 x 640 x 64, theta = 5 deg),
    all 3000 steps."""
    w = max(W.config4(), key=lambda x: x.cells)
    assert (w.nx, w.steps) == (640, 3000)
    errs = _f32_against_f64(w, (7, 16, 1))
    print(w.name, {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) <= TOL32, errs


def test_config2_first_600_steps_against_oracle():
    """The oracle over the first 600 steps of the 256 x 256 x 128 workload
    (about a minute on the host cores): FP64 to 1e-11, FP32 to 1e-4."""
    w = dataclasses.replace(W.config2(), steps=600)
    og, os_ = oracle_grid(w), oracle_source(w)
    st = oracle.State(og)
    oracle.run(og, os_, st, w.steps)
    for precision, tile, tol in (("f64", None, 1e-11), ("f32", (7, 16, 1), TOL32)):
        g = gpu_grid(w, precision, tile=tile)
        g.step(w.steps)
        errs = {n: rel_l2(host(g.field(c)), ref) for c, (n, ref) in enumerate(zip(NAMES, st.fields()))}
        errs["fluence"] = rel_l2(host(g.fluence()), st.fluence)
        print(w.name, precision, {k: f"{v:.2e}" for k, v in errs.items()})
        assert max(errs.values()) <= tol, (precision, errs)
        g.close()
