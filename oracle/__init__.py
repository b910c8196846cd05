"""FP64 CPU oracle of the Bessel-antenna FDTD (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The product path (the CUDA library and its
Python binding) never imports, links or runs anything here, and this package
imports nothing from the product.

The arithmetic lives in ``fdtd_oracle.c`` (plain C, FP64, one cell at a time);
this module compiles it with gcc, loads it with ctypes and converts between
NumPy arrays and the C structs.  What each C function follows in the paper is
stated in the C file's header and beside each function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

POL = {"y": 0, "x": 1, "circ+": 2, "circ-": 3, "z": 4}
MODE = {"TE": 0, "TM": 1}
ENV = {"cw": 0, "gauss": 1}
INJ = {"all": 0, "tangential": 1}


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library (gcc, -O2, OpenMP, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fPIC", "-shared",
           "-fopenmp", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("npml", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double), ("dt", C.c_double),
                ("pml_order", C.c_double), ("pml_sigma_scale", C.c_double),
                ("pml_kappa_max", C.c_double), ("pml_alpha_max", C.c_double),
                ("zbc", C.c_int), ("npml_z", C.c_int)]


class _Wall(C.Structure):
    _fields_ = [("theta", C.c_double), ("w0", C.c_double), ("E0", C.c_double), ("envelope", C.c_int),
                ("ramp", C.c_double), ("T", C.c_double), ("T0", C.c_double), ("plane", C.c_int)]


class _Source(C.Structure):
    _fields_ = [("m", C.c_int), ("theta", C.c_double), ("pol", C.c_int), ("mode", C.c_int),
                ("E0", C.c_double), ("r_center", C.c_double), ("thickness", C.c_double),
                ("envelope", C.c_int), ("ramp", C.c_double), ("T", C.c_double), ("T0", C.c_double),
                ("inject", C.c_int),
                ("w_amp", C.POINTER(C.c_double)), ("w_phase", C.POINTER(C.c_double))]


class _State(C.Structure):
    _fields_ = [("e", C.POINTER(C.c_double) * 3), ("h", C.POINTER(C.c_double) * 3),
                ("psi_e", C.POINTER(C.c_double) * 4), ("psi_h", C.POINTER(C.c_double) * 4),
                ("fluence", C.POINTER(C.c_double)),
                ("psi_ez", C.POINTER(C.c_double) * 2), ("psi_hz", C.POINTER(C.c_double) * 2)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            L.or_courant_dt.restype = C.c_double
            L.or_courant_dt.argtypes = [C.c_double] * 4
            L.or_jn.restype = C.c_double
            L.or_jn.argtypes = [C.c_int, C.c_double]
            L.or_pml_profile.restype = None
            L.or_pml_profile.argtypes = [C.POINTER(_Grid), C.c_int, C.c_double, C.c_double, dp, dp, dp]
            L.or_source_field.restype = None
            L.or_source_field.argtypes = [C.POINTER(_Source), C.c_double, C.c_double, C.c_double, dp, dp]
            L.or_bessel_pulse.restype = None
            L.or_bessel_pulse.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, C.c_double, C.c_long,
                                          dp, dp, dp, dp, C.c_int, dp]
            L.or_source_time.restype = None
            L.or_source_time.argtypes = [C.POINTER(_Source), C.c_double, dp, dp, dp]
            L.or_run.restype = C.c_int
            L.or_run.argtypes = [C.POINTER(_Grid), C.POINTER(_Source), C.POINTER(_State), C.c_long, C.c_int]
            L.or_run_wall.restype = C.c_int
            L.or_run_wall.argtypes = [C.POINTER(_Grid), C.POINTER(_Source), C.POINTER(_Wall), C.POINTER(_State),
                                      C.c_long, C.c_int]
            L.or_adjoint_step.restype = C.c_int
            L.or_adjoint_step.argtypes = [C.POINTER(_Grid), C.POINTER(_Source), C.POINTER(_State), C.c_long,
                                          dp, dp]
            L.or_threads.restype = C.c_int
            L.or_threads.argtypes = []
            L.or_set_threads.restype = None
            L.or_set_threads.argtypes = [C.c_int]
            L.or_antenna_counts.restype = C.c_int
            L.or_antenna_counts.argtypes = [C.POINTER(_Grid), C.POINTER(_Source), C.POINTER(C.c_long)]
            _lib = L
    return _lib


def threads() -> int:
    """OpenMP threads the oracle's loops use."""
    return int(lib().or_threads())


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))


def courant_dt(dx: float, dy: float, dz: float, courant: float) -> float:
    return lib().or_courant_dt(dx, dy, dz, courant)


def jn(n: int, x: float) -> float:
    return lib().or_jn(int(n), float(x))


@dataclass
class Grid:
    """Grid description (cells, cell sizes in wavelengths, CPML constants)."""
    nx: int
    ny: int
    nz: int
    npml: int
    dx: float
    dy: float
    dz: float
    courant: float = 0.95
    dt: float | None = None
    pml_order: float = 3.0
    pml_sigma_scale: float = 0.8
    pml_kappa_max: float = 1.0
    pml_alpha_max: float = 0.05 * 2.0 * np.pi
    z_walls: bool = False       # PEC walls at z = 0 and z = nz dz instead of periodic z
    npml_z: int = 0             # CPML cells inside each z wall (z_walls only)

    def __post_init__(self):
        if self.dt is None or self.dt == 0.0:
            self.dt = courant_dt(self.dx, self.dy, self.dz, self.courant)

    def _c(self) -> _Grid:
        return _Grid(self.nx, self.ny, self.nz, self.npml, self.dx, self.dy, self.dz, self.dt,
                     self.pml_order, self.pml_sigma_scale, self.pml_kappa_max, self.pml_alpha_max,
                     1 if self.z_walls else 0, self.npml_z if self.z_walls else 0)

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)


@dataclass
class Source:
    """Bessel-antenna description (ring radius and thickness in cells of dx)."""
    m: int = 0
    theta: float = np.deg2rad(20.0)
    pol: str = "y"
    mode: str = "TE"
    E0: float = 1.0
    r_center: float = 12.0
    thickness: float = 1.0
    envelope: str = "cw"
    ramp: float = 10.0
    T: float = 0.0
    T0: float = 0.0
    inject: str = "all"
    w_amp: np.ndarray | None = None
    w_phase: np.ndarray | None = None
    _keep: list = field(default_factory=list, repr=False)

    def _c(self) -> _Source:
        dp = C.POINTER(C.c_double)
        self._keep = []

        def arr(a):
            if a is None:
                return dp()
            a = np.ascontiguousarray(a, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(dp)

        return _Source(self.m, self.theta, POL[self.pol], MODE[self.mode], self.E0,
                       self.r_center, self.thickness, ENV[self.envelope], self.ramp, self.T,
                       self.T0, INJ[self.inject], arr(self.w_amp), arr(self.w_phase))


class State:
    """FP64 field state on the host: E at n dt, H at (n-1/2) dt, CPML psi, fluence."""

    def __init__(self, grid: Grid, fluence: bool = True):
        shp = grid.shape
        self.e = [np.zeros(shp) for _ in range(3)]
        self.h = [np.zeros(shp) for _ in range(3)]
        self.psi_e = [np.zeros(shp) for _ in range(4)]
        self.psi_h = [np.zeros(shp) for _ in range(4)]
        self.psi_ez = [np.zeros(shp) for _ in range(2)]
        self.psi_hz = [np.zeros(shp) for _ in range(2)]
        self.fluence = np.zeros(shp) if fluence else None
        self.n = 0

    def _c(self) -> _State:
        dp = C.POINTER(C.c_double)
        s = _State()
        for c in range(3):
            s.e[c] = self.e[c].ctypes.data_as(dp)
            s.h[c] = self.h[c].ctypes.data_as(dp)
        for c in range(4):
            s.psi_e[c] = self.psi_e[c].ctypes.data_as(dp)
            s.psi_h[c] = self.psi_h[c].ctypes.data_as(dp)
        s.fluence = self.fluence.ctypes.data_as(dp) if self.fluence is not None else dp()
        for c in range(2):
            s.psi_ez[c] = self.psi_ez[c].ctypes.data_as(dp)
            s.psi_hz[c] = self.psi_hz[c].ctypes.data_as(dp)
        return s

    def copy(self) -> "State":
        o = State.__new__(State)
        o.e = [a.copy() for a in self.e]
        o.h = [a.copy() for a in self.h]
        o.psi_e = [a.copy() for a in self.psi_e]
        o.psi_h = [a.copy() for a in self.psi_h]
        o.psi_ez = [a.copy() for a in self.psi_ez]
        o.psi_hz = [a.copy() for a in self.psi_hz]
        o.fluence = None if self.fluence is None else self.fluence.copy()
        o.n = self.n
        return o

    def fields(self):
        """(Ex, Ey, Ez, Hx, Hy, Hz) arrays, shape (nz, ny, nx)."""
        return (*self.e, *self.h)


@dataclass
class Wall:
    """Wall source (the Bessel-Gauss reference of Section 2): a Gaussian beam of
    waist w0 (wavelengths), polarised along x, with the axicon phase
    -k r sin(theta), added to E_x on plane `plane` after each E update."""
    theta: float = np.deg2rad(25.0)
    w0: float = 7.5
    E0: float = 1.0
    envelope: str = "cw"
    ramp: float = 10.0
    T: float = 0.0
    T0: float = 0.0
    plane: int = 0

    def _c(self) -> _Wall:
        return _Wall(self.theta, self.w0, self.E0, ENV[self.envelope], self.ramp, self.T, self.T0, self.plane)


def run(grid: Grid, source: Source | None, state: State, nsteps: int, wall: Wall | None = None) -> State:
    """Advance `state` by nsteps Yee steps in place (Section 4, Eq. 13; the
    wall source of Section 2 if given)."""
    for a in (*state.e, *state.h, *state.psi_e, *state.psi_h, *state.psi_ez, *state.psi_hz):
        assert a.flags.c_contiguous and a.dtype == np.float64 and a.shape == grid.shape
    g = grid._c()
    s = source._c() if source is not None else None
    w = wall._c() if wall is not None else None
    st = state._c()
    rc = lib().or_run_wall(C.byref(g), C.byref(s) if s is not None else None,
                           C.byref(w) if w is not None else None, C.byref(st), state.n, int(nsteps))
    if rc != 0:
        raise RuntimeError(f"oracle run failed ({rc})")
    state.n += nsteps
    return state


def adjoint_step(grid: Grid, source: Source | None, adj: State, n: int, grad_amp=None, grad_phase=None):
    """One reverse step: the exact transpose of forward step n applied to the
    adjoint state `adj` (adjoints of E^{n+1}, H^{n+1/2}, psi on entry; of
    E^n, H^{n-1/2}, psi on return).  grad_amp / grad_phase (ny, nx) arrays
    accumulate dL/dw of the source terms of step n."""
    dp = C.POINTER(C.c_double)
    g = grid._c()
    s = source._c() if source is not None else None
    st = adj._c()
    ga = grad_amp.ctypes.data_as(dp) if grad_amp is not None else dp()
    gp = grad_phase.ctypes.data_as(dp) if grad_phase is not None else dp()
    rc = lib().or_adjoint_step(C.byref(g), C.byref(s) if s is not None else None, C.byref(st), int(n), ga, gp)
    if rc != 0:
        raise RuntimeError("oracle adjoint step failed")
    return adj


def bessel_pulse(m: int, theta: float, T: float, T0: float, r, phi, z, t, w0: float = 2 * np.pi,
                 nq: int = 4001) -> np.ndarray:
    """Complex E_y of the order-m Bessel pulse of Eq. 11 (Gaussian spectrum of
    Eq. 10, width T and peak time T0 in periods, centre w0) at the broadcast
    points (r, phi, z, t), by quadrature, in the e^{-i w t} convention of the
    source fields: the physical field is the real part."""
    r, phi, z, t = np.broadcast_arrays(*(np.asarray(a, dtype=np.float64) for a in (r, phi, z, t)))
    shape = r.shape
    cols = [np.ascontiguousarray(a.ravel()) for a in (r, phi, z, t)]
    out = np.zeros(2 * cols[0].size)
    dp = C.POINTER(C.c_double)
    lib().or_bessel_pulse(int(m), float(theta), float(T), float(T0), float(w0), cols[0].size,
                          *(a.ctypes.data_as(dp) for a in cols), int(nq), out.ctypes.data_as(dp))
    return (out[0::2] + 1j * out[1::2]).reshape(shape)


def source_field(source: Source, x: float, y: float, z: float):
    """Complex amplitudes (E[3], H[3]) of the analytic beam at (x, y, z) from the axis."""
    E = (C.c_double * 6)()
    H = (C.c_double * 6)()
    s = source._c()
    lib().or_source_field(C.byref(s), x, y, z, E, H)
    e = np.array([E[0] + 1j * E[1], E[2] + 1j * E[3], E[4] + 1j * E[5]])
    h = np.array([H[0] + 1j * H[1], H[2] + 1j * H[3], H[4] + 1j * H[5]])
    return e, h


def source_time(source: Source, t: float):
    """(cos Phi, sin Phi, f) of the soft source at time t."""
    c, s, f = C.c_double(), C.c_double(), C.c_double()
    src = source._c()
    lib().or_source_time(C.byref(src), t, C.byref(c), C.byref(s), C.byref(f))
    return c.value, s.value, f.value


def pml_profile(grid: Grid, axis_n: int, d: float, pos: float):
    b, a, k = C.c_double(), C.c_double(), C.c_double()
    g = grid._c()
    lib().or_pml_profile(C.byref(g), axis_n, d, pos, C.byref(b), C.byref(a), C.byref(k))
    return b.value, a.value, k.value


def antenna_counts(grid: Grid, source: Source):
    cnt = (C.c_long * 6)()
    g = grid._c()
    s = source._c()
    if lib().or_antenna_counts(C.byref(g), C.byref(s), cnt) != 0:
        raise RuntimeError("antenna build failed")
    return [int(c) for c in cnt]
