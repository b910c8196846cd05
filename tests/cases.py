"""Adapters from a workload recipe to the oracle's descriptors (tests only)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2102_12978_gb300.workloads import WallWorkload, Workload


def oracle_grid(w: Workload, npml: int | None = None) -> oracle.Grid:
    return oracle.Grid(w.nx, w.ny, w.nz, w.npml if npml is None else npml,
                       w.dx, w.dx, w.dz, courant=w.courant)


def oracle_source(w: Workload, w_amp=None, w_phase=None) -> oracle.Source:
    return oracle.Source(m=w.m, theta=w.theta, pol=w.pol, mode=w.mode, E0=w.E0,
                         r_center=w.r_center, thickness=w.thickness, envelope=w.envelope,
                         ramp=w.ramp, T=w.T, T0=w.T0, inject=w.inject,
                         w_amp=w_amp, w_phase=w_phase)


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b.ravel())
    num = np.linalg.norm((a - b).ravel())
    return float(num / den) if den > 0 else float(num)


def oracle_wall_grid(w: WallWorkload, z_walls: bool = True) -> oracle.Grid:
    """The recipe's z-walled box with its z CPML, or (z_walls=False) the same
    box periodic in z."""
    return oracle.Grid(w.nx, w.ny, w.nz, w.npml, w.dx, w.dx, w.dz, courant=w.courant, z_walls=z_walls,
                       npml_z=w.npml_z if z_walls else 0)


def oracle_wall(w: WallWorkload) -> oracle.Wall:
    return oracle.Wall(theta=w.theta, w0=w.w0, E0=w.E0, envelope=w.envelope, ramp=w.ramp, T=w.T, T0=w.T0,
                       plane=w.plane)
