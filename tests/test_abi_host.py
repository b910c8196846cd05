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


def test_invalid_z_boundaries_rejected():
    kw = dict(nx=32, ny=32, nz=16, npml=6, dx=0.05, dy=0.05, dz=0.05)
    assert fdtd.fdtd_required_bytes(fdtd.make_grid_desc(**kw, z_walls=True, npml_z=7)) > 0
    assert fdtd.fdtd_required_bytes(fdtd.make_grid_desc(**kw, z_walls=True, npml_z=0)) > 0
    for bad in [dict(z_walls=True, npml_z=8), dict(z_walls=True, npml_z=-1), dict(z_walls=False, npml_z=2)]:
        assert fdtd.fdtd_required_bytes(fdtd.make_grid_desc(**kw, **bad)) == 0, bad
    d = fdtd.make_grid_desc(**kw)
    d.z_boundary = 2
    assert fdtd.fdtd_required_bytes(d) == 0
    # tall z-walled grids are taken (the cell passes launch chunks of planes)
    assert fdtd.fdtd_required_bytes(fdtd.make_grid_desc(4, 4, 70000, 0, 0.05, 0.05, 0.05, z_walls=True)) > 0
    # the z shell adds its psi arrays to the arena
    a = fdtd.fdtd_required_bytes(fdtd.make_grid_desc(**kw, z_walls=True, npml_z=4))
    b = fdtd.fdtd_required_bytes(fdtd.make_grid_desc(**kw, z_walls=True, npml_z=0))
    assert a > b


def test_antenna_rejected_on_z_walls():
    """The antenna boxes are z-periodic (Section 4): both sides refuse an
    antenna on a z-walled grid."""
    d = fdtd.make_grid_desc(40, 40, 16, 6, 1 / 16, 1 / 16, 1 / 16, z_walls=True, npml_z=4)
    s, _ = fdtd.make_annulus_desc(r_center=9.0)
    with pytest.raises(fdtd.FDTDError) as e:
        fdtd.source_coefficients(d, s)
    assert e.value.status == fdtd.FDTD_EINVAL
    g = oracle.Grid(40, 40, 16, 6, 1 / 16, 1 / 16, 1 / 16, z_walls=True, npml_z=4)
    with pytest.raises(RuntimeError):
        oracle.run(g, oracle.Source(r_center=9.0), oracle.State(g), 1)


@pytest.mark.parametrize("z_walls", [False, True])
def test_wall_coefficients_match_oracle_sheet(z_walls):
    """The library's FP64 wall coefficients W (Section 2: Gaussian waist times
    the axicon phase) against the oracle's own sheet: one oracle step from
    zero fields leaves E_x = f Re{W e^{-i Phi}} on the sheet plane.  A
    Gaussian envelope with T0 = dt gives Phi = 0 (Re W), with T0 = dt - 1/4
    gives Phi = pi/2 (Im W); f is divided out."""
    nx, ny, nz, dx = 37, 30, 12, 1 / 16
    th, w0, E0, plane = np.deg2rad(25.0), 0.7, 1.3, 5
    d = fdtd.make_grid_desc(nx, ny, nz, 4, dx, dx, dx, z_walls=z_walls, npml_z=2 if z_walls else 0)
    Wl = fdtd.wall_coefficients(d, fdtd.make_wall_desc(theta=th, w0=w0, E0=E0, envelope="gauss", T=1.0,
                                                       T0=0.0, plane=plane))
    assert np.all(Wl[0] == 0)
    g = oracle.Grid(nx, ny, nz, 4, dx, dx, dx, z_walls=z_walls, npml_z=2 if z_walls else 0)
    got = []
    for shift in (0.0, 0.25):
        T = 50.0
        wall = oracle.Wall(theta=th, w0=w0, E0=E0, envelope="gauss", T=T, T0=g.dt - shift, plane=plane)
        st = oracle.State(g, fluence=False)
        oracle.run(g, None, st, 1, wall=wall)
        f = math.exp(-(shift / T) ** 2)
        got.append(st.e[0][plane] / f)
        assert np.count_nonzero(st.e[0][np.arange(nz) != plane]) == 0
    ref = got[0] + 1j * got[1]
    np.testing.assert_allclose(Wl.real, ref.real, rtol=0, atol=1e-14 * E0)
    np.testing.assert_allclose(Wl.imag, ref.imag, rtol=0, atol=1e-14 * E0)
    # the waist: |W| = E0 exp(-r^2/w0^2) at the E_x points
    x = (np.arange(nx) + 0.5 - nx / 2) * dx
    y = (np.arange(ny) - ny / 2) * dx
    r2 = x[None, :] ** 2 + y[:, None] ** 2
    np.testing.assert_allclose(np.abs(Wl[1:]), (E0 * np.exp(-r2 / w0 ** 2))[1:], rtol=1e-14, atol=0)


def test_invalid_wall_descriptors_rejected():
    d = fdtd.make_grid_desc(32, 32, 16, 6, 0.05, 0.05, 0.05, z_walls=True, npml_z=4)
    out = np.zeros(2 * 32 * 32)
    for bad in [dict(w0=0.0), dict(plane=16), dict(plane=-1), dict(plane=0), dict(envelope="gauss", T=0.0),
                dict(ramp=-1.0)]:
        w = fdtd.make_wall_desc(**{**dict(plane=5), **bad})
        assert fdtd.lib().fdtd_wall_coefficients(fdtd.C.byref(d), fdtd.C.byref(w), out.ctypes.data) \
            == fdtd.FDTD_EINVAL, bad
    # plane 0 is allowed on a z-periodic grid
    dp = fdtd.make_grid_desc(32, 32, 16, 6, 0.05, 0.05, 0.05)
    w = fdtd.make_wall_desc(plane=0)
    assert fdtd.lib().fdtd_wall_coefficients(fdtd.C.byref(dp), fdtd.C.byref(w), out.ctypes.data) == fdtd.FDTD_OK
