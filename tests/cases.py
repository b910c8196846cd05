"""Adapters from a workload recipe to the oracle's descriptors (tests only)."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2102_12978_gb300.workloads import Workload


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
