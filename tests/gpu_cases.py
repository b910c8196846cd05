"""Helpers for the GPU tests: build a library grid from a workload recipe."""
from __future__ import annotations

import numpy as np

from paper_2102_12978_gb300 import fdtd
from paper_2102_12978_gb300.workloads import WallWorkload, Workload


def gpu_grid(w: Workload, precision: str = "f64", fluence: bool = True, npml: int | None = None,
             source: bool = True, w_amp=None, w_phase=None, tile=None) -> fdtd.Grid:
    d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml if npml is None else npml, w.dx, w.dx, w.dz,
                            courant=w.courant, precision=precision, fluence=fluence)
    g = fdtd.Grid(d)
    if tile is not None:
        g.set_tile(*tile)
    if source:
        g.set_source(m=w.m, theta=w.theta, pol=w.pol, mode=w.mode, E0=w.E0, r_center=w.r_center,
                     thickness=w.thickness, envelope=w.envelope, ramp=w.ramp, T=w.T, T0=w.T0,
                     inject=w.inject, w_amp=w_amp, w_phase=w_phase)
    return g


def host(t) -> np.ndarray:
    return t.detach().to("cpu").double().numpy()


def gpu_wall_grid(w: WallWorkload, precision: str = "f64", fluence: bool = True, wall: bool = True,
                  tile=None, z_walls: bool = True) -> fdtd.Grid:
    """A library grid for a Bessel-Gauss recipe: z walls with the recipe's z
    CPML (or, z_walls=False, a z-periodic box) and the wall sheet."""
    d = fdtd.make_grid_desc(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant,
                            precision=precision, fluence=fluence, z_walls=z_walls,
                            npml_z=w.npml_z if z_walls else 0)
    g = fdtd.Grid(d)
    if tile is not None:
        g.set_tile(*tile)
    if wall:
        g.set_wall_source(theta=w.theta, w0=w.w0, E0=w.E0, envelope=w.envelope, ramp=w.ramp, T=w.T,
                          T0=w.T0, plane=w.plane)
    return g
