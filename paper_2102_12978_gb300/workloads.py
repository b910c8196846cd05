"""Seeded synthetic workloads: grid shapes, beam parameters and random inputs.

This module holds no arithmetic of the method.  It only states the workload
recipes (box sizes, cell sizes, cone angles, ring radii, step counts) and the
seeded random generators, so that the CUDA path and the CPU oracle are fed the
same inputs.  Units: lengths in source wavelengths (lambda = 1, i.e. 0.8 um in
the paper's SI setup), times in optical periods; ring radius and thickness in
cells of dx.

The shapes follow the paper's own setups (Section 4: a box spanning an integer
number of axial periods lambda_z = lambda / cos(theta) so that z is periodic, a
cubic-ish mesh of 16-24 cells per wavelength, a CPML shell on the transverse
faces, and a hollow annulus well inside the PML-free region) at the sizes of
the benchmark configurations below.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

SEED = 20260101


def rng(seed: int = SEED) -> np.random.Generator:
    """PCG64 generator used for every random input (weights, states)."""
    return np.random.Generator(np.random.PCG64(seed))


def dz_for_periods(nz: int, dx: float, theta_deg: float, periods: int | None = None) -> float:
    """Cell size along z so that nz cells span exactly `periods` axial periods.

    If `periods` is None it is the integer nearest to nz*dx / lambda_z, which
    keeps dz close to dx (Section 4 sampling rule, made exactly periodic)."""
    lam_z = 1.0 / math.cos(math.radians(theta_deg))
    if periods is None:
        periods = max(1, round(nz * dx / lam_z))
    return periods * lam_z / nz


@dataclass
class Workload:
    """One single-beam configuration."""
    name: str
    nx: int
    ny: int
    nz: int
    npml: int
    dx: float
    dz: float
    theta_deg: float
    m: int
    pol: str                 # "y" (Pi_x potential), "x" (Pi_y), "circ+", "circ-"
    r_center: float          # cells
    thickness: float         # cells
    steps: int
    ramp: float = 10.0       # sin^2 ramp of the CW envelope, periods
    courant: float = 0.95
    inject: str = "all"
    mode: str = "TE"
    envelope: str = "cw"
    T: float = 0.0
    T0: float = 0.0
    E0: float = 1.0
    extra: dict = field(default_factory=dict)

    @property
    def theta(self) -> float:
        return math.radians(self.theta_deg)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def scaled(self, **kw) -> "Workload":
        return replace(self, **kw)


def _interior_ring(n: int, npml: int, frac: float = 0.8) -> float:
    return frac * (n - 2 * npml) / 2.0


def config1() -> Workload:
    """64x64x32, dx = lambda/16, 2 axial periods in z, theta = 20 deg, l = 0,
    x-polarised, tangential injection on a 1-cell ring of radius 12 cells,
    8-cell CPML, 400 steps."""
    nz, dx, th = 32, 1.0 / 16, 20.0
    return Workload("cfg1_64x64x32_f64", 64, 64, nz, 8, dx, dz_for_periods(nz, dx, th, 2), th,
                    0, "x", 12.0, 1.0, 400, inject="tangential")


def config2() -> Workload:
    """256x256x128, dx = lambda/20, theta = 10 deg, l = 0, ring radius 100
    cells, 16-cell CPML, 4000 steps."""
    nz, dx, th = 128, 1.0 / 20, 10.0
    return Workload("cfg2_256x256x128", 256, 256, nz, 16, dx, dz_for_periods(nz, dx, th), th,
                    0, "y", 100.0, 1.0, 4000)


def config3() -> list[Workload]:
    """512x512x64, dx = lambda/24, l in {1,2,3} x theta in {15,30}, plus the
    circular l = 1 variant; ring radius 0.8 x interior half-width; 6000 steps."""
    out = []
    nz, dx, n, npml = 64, 1.0 / 24, 512, 16
    for th in (15.0, 30.0):
        for m in (1, 2, 3):
            out.append(Workload(f"cfg3_m{m}_t{int(th)}", n, n, nz, npml, dx,
                                dz_for_periods(nz, dx, th), th, m, "y",
                                _interior_ring(n, npml), 1.0, 6000))
    out.append(Workload("cfg3_circ_m1_t15", n, n, nz, npml, dx, dz_for_periods(nz, dx, 15.0), 15.0,
                        1, "circ+", _interior_ring(n, npml), 1.0, 6000))
    return out


def config4() -> list[Workload]:
    """Batched sweep: l in {0..3} x theta in {5,10,20,30} deg; transverse size
    N = 32 round(8 r0 / (32 dx)), r0 = 0.383 lambda / sin(theta), dx = lambda/18,
    N x N x 64 cells, 16-cell CPML, 3000 steps each."""
    out = []
    dx, nz, npml = 1.0 / 18, 64, 16
    for th in (5.0, 10.0, 20.0, 30.0):
        r0 = 0.383 / math.sin(math.radians(th))
        n = 32 * round(8 * r0 / (32 * dx))
        for m in range(4):
            out.append(Workload(f"cfg4_m{m}_t{int(th)}_{n}", n, n, nz, npml, dx,
                                dz_for_periods(nz, dx, th), th, m, "y",
                                _interior_ring(n, npml), 1.0, 3000))
    return out


def config5() -> Workload:
    """Adjoint workload: 384x384x96, dx = lambda/20, theta = 15 deg, l = 0,
    ring 0.8 x interior half-width, 3 cells thick, 5000 steps."""
    nz, dx, th, n, npml = 96, 1.0 / 20, 15.0, 384, 16
    return Workload("cfg5_384x384x96", n, n, nz, npml, dx, dz_for_periods(nz, dx, th), th,
                    0, "y", _interior_ring(n, npml), 3.0, 5000)


def small(name: str = "small", nx: int = 48, ny: int = 40, nz: int = 16, npml: int = 6,
          theta_deg: float = 20.0, m: int = 0, pol: str = "y", r_center: float = 10.0,
          thickness: float = 1.0, steps: int = 60, dx: float = 1.0 / 16, **kw) -> Workload:
    """A small case the oracle finishes in about a second, still spanning
    several tiles and ragged tile tails."""
    return Workload(name, nx, ny, nz, npml, dx, dz_for_periods(nz, dx, theta_deg), theta_deg,
                    m, pol, r_center, thickness, steps, **kw)


# One optical period at the paper's lambda = 0.8 um, in femtoseconds.
FS_PER_PERIOD = 0.8e-6 / 299792458.0 * 1e15


@dataclass
class WallWorkload:
    """One Bessel-Gauss configuration (Section 2): a z-walled box, CPML on
    all six faces, and the Gaussian-times-axicon E_x sheet on plane `plane`."""
    name: str
    nx: int
    ny: int
    nz: int
    npml: int                # transverse CPML cells
    npml_z: int              # CPML cells inside each z wall
    dx: float
    dz: float
    theta_deg: float         # axicon cone angle
    w0: float                # Gaussian waist, wavelengths
    plane: int               # E plane of the sheet
    steps: int
    envelope: str = "gauss"
    T: float = 0.0           # Gaussian envelope exp(-(t-T0)^2/T^2), periods
    T0: float = 0.0
    ramp: float = 0.0        # CW ramp, periods
    courant: float = 0.95
    E0: float = 1.0

    @property
    def theta(self) -> float:
        return math.radians(self.theta_deg)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    def scaled(self, **kw) -> "WallWorkload":
        return replace(self, **kw)


def bessel_gauss() -> WallWorkload:
    """The Bessel-Gauss box of Section 2: lambda = 0.8 um, theta = 25 deg, an
    8 lambda_xy x 8 lambda_xy x 32 lambda_z interior (lambda_xy = lambda /
    sin(theta), lambda_z = lambda / cos(theta); 15 x 15 x 28 um), waist
    w0 = 6 um, a Gaussian amplitude of 100 fs FWHM (T = FWHM / (2 sqrt(ln 2)))
    centred at T0 = 2 T, run to t_run = 266 fs.  Mesh (not given for this
    run): dx = dz = lambda/20, 16 CPML cells on every face, Courant 0.95 of
    the cubic Yee limit; the sheet sits on the first plane past the low-z
    CPML (k = 16).  Interior 379 x 379 x 706 cells, 411 x 411 x 738 with the CPML."""
    th, dx, npml = 25.0, 1.0 / 20, 16
    lam_xy = 1.0 / math.sin(math.radians(th))
    lam_z = 1.0 / math.cos(math.radians(th))
    n_in = round(8 * lam_xy / dx)
    nz_in = round(32 * lam_z / dx)
    T = (100.0 / FS_PER_PERIOD) / (2.0 * math.sqrt(math.log(2.0)))
    courant = 0.95
    dt = courant * dx / math.sqrt(3.0)
    steps = math.ceil((266.0 / FS_PER_PERIOD) / dt)
    return WallWorkload("bessel_gauss_411x411x738", n_in + 2 * npml, n_in + 2 * npml, nz_in + 2 * npml,
                        npml, npml, dx, dx, th, 6.0 / 0.8, npml, steps, envelope="gauss", T=T, T0=2 * T,
                        courant=courant)


def small_wall(name: str = "small_wall", nx: int = 40, ny: int = 36, nz: int = 32, npml: int = 6,
               npml_z: int = 6, theta_deg: float = 25.0, w0: float = 0.6, plane: int | None = None,
               steps: int = 60, dx: float = 1.0 / 16, **kw) -> WallWorkload:
    """A small z-walled case the oracle finishes in about a second."""
    return WallWorkload(name, nx, ny, nz, npml, npml_z, dx, dx, theta_deg, w0,
                        npml_z + 1 if plane is None else plane, steps, **kw)


def random_state(shape, scale: float = 1.0, seed: int = SEED):
    """Six seeded random field arrays (Ex, Ey, Ez, Hx, Hy, Hz), FP64."""
    g = rng(seed)
    return [scale * g.standard_normal(shape) for _ in range(6)]


def random_weights(nx: int, ny: int, seed: int = SEED, amp_sigma: float = 0.1,
                   phase_sigma: float = 0.1):
    """Seeded per-column amplitude and phase weights around (1, 0)."""
    g = rng(seed)
    amp = 1.0 + amp_sigma * g.standard_normal((ny, nx))
    ph = phase_sigma * g.standard_normal((ny, nx))
    return amp, ph
