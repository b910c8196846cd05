"""Parity at the full sizes of the benchmark configurations, in the launch
configuration the bench times (cell-parallel passes, 32 x 4 blocks; the
batched sweep's default engine): the first steps of each configuration --
long enough for the antenna's field to cross many tiles -- element by element
against the FP64 oracle on the whole grid.  The oracle runs these sizes in
seconds on the host cores (OpenMP over z planes)."""
import dataclasses

import numpy as np
import pytest

import oracle
from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300 import workloads as W
from tests.cases import oracle_grid, oracle_source, rel_l2
from tests.gpu_cases import gpu_grid, host

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-11, "f32": 1e-4}
BENCH_TILE = (5, 4, 1)


def _oracle_run(w):
    og, os_ = oracle_grid(w), oracle_source(w)
    st = oracle.State(og)
    oracle.run(og, os_, st, w.steps)
    return st


def _check(g, st, precision, name):
    errs = {}
    for c, ref in enumerate(st.fields()):
        errs["ExEyEzHxHyHz"[2 * c:2 * c + 2]] = rel_l2(host(g.field(c)), ref)
    errs["fluence"] = rel_l2(host(g.fluence()), st.fluence)
    print(name, precision, {k: f"{v:.2e}" for k, v in errs.items()})
    bad = {k: v for k, v in errs.items() if not (v <= TOL[precision])}
    assert not bad, (name, precision, errs)


@pytest.mark.parametrize("precision", ["f32", "f64"])
def test_config2_full_size(precision):
    """256x256x128, the bench workload, 40 steps."""
    w = dataclasses.replace(W.config2(), steps=40)
    g = gpu_grid(w, precision, tile=BENCH_TILE)
    g.step(w.steps)
    g.sync()
    _check(g, _oracle_run(w), precision, w.name)


def test_config3_full_size_f32():
    """512x512x64, l = 2, theta = 30 deg, 40 steps."""
    w = dataclasses.replace(W.config3()[4], steps=40)
    assert (w.m, w.theta_deg) == (2, 30.0)
    g = gpu_grid(w, "f32", tile=BENCH_TILE)
    g.step(w.steps)
    g.sync()
    _check(g, _oracle_run(w), "f32", w.name)


def test_config5_full_size_f32():
    """384x384x96 with the 3-cell-thick ring, 40 steps."""
    w = dataclasses.replace(W.config5(), steps=40)
    g = gpu_grid(w, "f32", tile=BENCH_TILE)
    g.step(w.steps)
    g.sync()
    _check(g, _oracle_run(w), "f32", w.name)


def test_config4_batched_full_size_f32():
    """The 16-grid sweep batched (default engine), 30 steps; three of its
    grids (N = 96, l = 3; N = 160, l = 1; N = 320, l = 2) against the oracle."""
    ws = [dataclasses.replace(w, steps=30) for w in W.config4()]
    grids = [gpu_grid(w, "f32") for w in ws]
    b = fdtd.Batch(grids)
    assert b.engine == fdtd.BATCH_CELL
    b.step(30)
    b.sync()
    keys = [(w.nx, w.m) for w in ws]
    for key in ((96, 3), (160, 1), (320, 2)):
        q = keys.index(key)
        _check(grids[q], _oracle_run(ws[q]), "f32", ws[q].name)
    b.close()


def test_largest_grid_keeps_every_plane_exact():
    """The largest grid the library takes: 2048 x 2048 x 503 FP32 cells, each
    array just under its 2^31-element bound (about 140 GB on the device).
    A z-independent state stays z-independent in a z-periodic box (every z
    difference is exactly zero), so after 3 steps every plane of the fields
    and of the fluence must equal, bit for bit, the single plane of the same
    run on a one-plane grid: a wrong index anywhere up to the last plane
    breaks that."""
    import torch
    nx, ny, nz, npml = 2048, 2048, 503, 16
    d = fdtd.make_grid_desc(nx, ny, nz, npml, 1 / 20, 1 / 20, 1 / 20, precision="f32", fluence=True)
    need = fdtd.fdtd_required_bytes(d) + 2 * nz * ny * nx * 8   # arena, one field copy, the FP64 fluence export
    if torch.cuda.mem_get_info()[0] < need:
        pytest.skip(f"needs {need / 1e9:.0f} GB of free device memory")
    assert float(nz) * ny * (nx + 31) < 2 ** 31            # the library's bound, with room for the pitch
    gen = torch.Generator().manual_seed(W.SEED + 31)
    base = [torch.randn(ny, nx, generator=gen) for _ in range(6)]
    base[1][:, 0] = 0; base[2][:, 0] = 0                    # tangential E on the i = 0 wall
    base[0][0, :] = 0; base[2][0, :] = 0                    # and on the j = 0 wall
    small = fdtd.Grid(fdtd.make_grid_desc(nx, ny, 1, npml, 1 / 20, 1 / 20, 1 / 20, precision="f32", fluence=True))
    for c in range(6):
        small.set_field(c, base[c][None])
    small.step(3)
    ref = [small.field(c)[0] for c in range(6)] + [small.fluence()[0]]
    big = fdtd.Grid(d)
    for c in range(6):
        big.set_field(c, base[c].cuda()[None].expand(nz, ny, nx))
    big.step(3)
    big.sync()
    for c in range(6):
        f = big.field(c)
        assert torch.equal(f, ref[c][None].expand_as(f)), c
        del f
        torch.cuda.empty_cache()
    F = big.fluence()
    assert torch.equal(F, ref[6][None].expand_as(F))
    del F
    big.close()
    small.close()
    torch.cuda.empty_cache()
