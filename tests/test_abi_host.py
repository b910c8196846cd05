"""CPU-side checks of the C-ABI library: it builds, loads, exports every
symbol include/fdtd.h declares, rejects bad descriptors, and its host FP64
precompute (its own Bessel routine and a gradient/Hessian form of Q and R)
agrees with the oracle's independent transcription of Eq. 6-9.  No kernel is
launched here."""
import math
import os
import re

import numpy as np
import pytest
from scipy import special

import oracle
from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(fdtd_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = fdtd.lib()
    names = _declared_symbols()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_bessel_recurrence_matches_scipy():
    xs = np.concatenate([np.linspace(0, 3, 31), np.linspace(3, 45, 85)])
    for n in range(-4, 8):
        got = np.array([fdtd.fdtd_bessel_j(n, x) for x in xs])
        np.testing.assert_allclose(got, special.jv(n, xs), rtol=0, atol=2e-15)


def test_invalid_descriptors_rejected():
    d = fdtd.make_grid_desc(32, 32, 8, 6, 0.05, 0.05, 0.05)
    assert fdtd.fdtd_required_bytes(d) > 0
    bad = [dict(courant=1.5), dict(npml=20), dict(nx=1), dict(dx=-1.0)]
    for b in bad:
        kw = dict(nx=32, ny=32, nz=8, npml=6, dx=0.05, dy=0.05, dz=0.05)
        kw.update(b)
        d = fdtd.make_grid_desc(**kw)
        assert fdtd.fdtd_required_bytes(d) == 0, b
    # create_grid refuses a null arena without touching a device
    d = fdtd.make_grid_desc(32, 32, 8, 6, 0.05, 0.05, 0.05)
    with pytest.raises(fdtd.FDTDError) as e:
        fdtd.fdtd_create_grid(d, 0, fdtd.fdtd_required_bytes(d), 0)
    assert e.value.status == fdtd.FDTD_EINVAL


OFF = [(0.5, 0, 0), (0, 0.5, 0), (0, 0, 0.5), (0, 0.5, 0.5), (0.5, 0, 0.5), (0.5, 0.5, 0)]


@pytest.mark.parametrize("m,pol,mode,inject", [(0, "y", "TE", "all"), (1, "x", "TE", "all"),
                                               (2, "circ+", "TE", "all"), (3, "y", "TM", "tangential"),
                                               (1, "circ-", "TM", "all"), (0, "z", "TE", "all"),
                                               (0, "z", "TM", "all"), (2, "z", "TM", "tangential")])
def test_host_precompute_matches_oracle_fields(m, pol, mode, inject):
    """A_c at every antenna column: library precompute vs oracle (FP64)."""
    w = W.small(nx=40, ny=36, nz=8, npml=4, theta_deg=23.0, m=m, pol=pol, r_center=9.0,
                thickness=2.0, mode=mode, inject=inject)
    d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz)
    s, _ = fdtd.make_annulus_desc(m=m, theta=w.theta, pol=pol, mode=mode, r_center=w.r_center,
                                  thickness=w.thickness, inject=inject)
    coef, mask = fdtd.source_coefficients(d, s)
    src = oracle.Source(m=m, theta=w.theta, pol=pol, mode=mode, r_center=w.r_center,
                        thickness=w.thickness, inject=inject)
    n_pts = 0
    for c in range(6):
        js, is_ = np.nonzero(mask & (1 << c))
        assert len(js) > 0
        for j, i in zip(js, is_):
            x = (i + OFF[c][0] - w.nx / 2) * w.dx
            y = (j + OFF[c][1] - w.ny / 2) * w.dx
            z = OFF[c][2] * w.dz
            e, h = oracle.source_field(src, x, y, z)
            ref = e[c] if c < 3 else h[c - 3]
            assert abs(coef[c, j, i] - ref) < 1e-13 * (1 + abs(ref)), (c, i, j)
            n_pts += 1
        # no coefficient outside the mask
        assert np.all(coef[c][(mask & (1 << c)) == 0] == 0)
    # the antenna point count agrees with the oracle's enumeration
    g = oracle.Grid(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz)
    counts = oracle.antenna_counts(g, src)
    lib_counts = [int(np.count_nonzero(mask & (1 << c))) * w.nz for c in range(6)]
    assert counts == lib_counts
