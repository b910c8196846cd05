"""Thin Python binding of libfdtd_gb300.so (include/fdtd.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device arena (a uint8 tensor) and the CUDA
stream.  If the library cannot be built or loaded this module raises; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

FDTD_OK, FDTD_EINVAL, FDTD_ENOMEM, FDTD_ECUDA, FDTD_ETIMEOUT, FDTD_ESTATE = range(6)
FDTD_F32, FDTD_F64 = 0, 1
EX, EY, EZ, HX, HY, HZ = range(6)
POL = {"y": 0, "x": 1, "circ+": 2, "circ-": 3, "z": 4}
MODE = {"TE": 0, "TM": 1}
ENV = {"cw": 0, "gauss": 1}
INJ = {"all": 0, "tangential": 1}


class FDTDError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str):
        super().__init__(f"{where}: status {status} ({detail})")
        self.status = status


class fdtd_grid_desc(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("npml", C.c_int),
                ("dx", C.c_double), ("dy", C.c_double), ("dz", C.c_double),
                ("dt", C.c_double), ("courant", C.c_double),
                ("pml_order", C.c_double), ("pml_sigma_scale", C.c_double),
                ("pml_kappa_max", C.c_double), ("pml_alpha_max", C.c_double),
                ("precision", C.c_int), ("fluence", C.c_int),
                ("z_boundary", C.c_int), ("npml_z", C.c_int)]


FDTD_Z_PERIODIC, FDTD_Z_WALLS = 0, 1


class fdtd_wall_desc(C.Structure):
    _fields_ = [("theta", C.c_double), ("w0", C.c_double), ("E0", C.c_double), ("envelope", C.c_int),
                ("ramp", C.c_double), ("T", C.c_double), ("T0", C.c_double), ("plane", C.c_int)]


class fdtd_annulus_desc(C.Structure):
    _fields_ = [("m", C.c_int), ("theta", C.c_double), ("pol", C.c_int), ("mode", C.c_int),
                ("E0", C.c_double), ("r_center", C.c_double), ("thickness", C.c_double),
                ("envelope", C.c_int), ("ramp", C.c_double), ("T", C.c_double), ("T0", C.c_double),
                ("inject", C.c_int),
                ("w_amp", C.POINTER(C.c_double)), ("w_phase", C.POINTER(C.c_double))]


_SIGS = {
    "fdtd_grid_desc_default": (None, [C.POINTER(fdtd_grid_desc)]),
    "fdtd_required_bytes": (C.c_size_t, [C.POINTER(fdtd_grid_desc)]),
    "fdtd_create_grid": (C.c_int, [C.POINTER(fdtd_grid_desc), C.c_void_p, C.c_size_t, C.c_void_p,
                                   C.POINTER(C.c_void_p)]),
    "fdtd_set_annulus_source": (C.c_int, [C.c_void_p, C.POINTER(fdtd_annulus_desc)]),
    "fdtd_clear_source": (C.c_int, [C.c_void_p]),
    "fdtd_set_wall_source": (C.c_int, [C.c_void_p, C.POINTER(fdtd_wall_desc)]),
    "fdtd_wall_coefficients": (C.c_int, [C.POINTER(fdtd_grid_desc), C.POINTER(fdtd_wall_desc), C.c_void_p]),
    "fdtd_step": (C.c_int, [C.c_void_p, C.c_int]),
    "fdtd_fluence": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "fdtd_get_field": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "fdtd_set_field": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int]),
    "fdtd_state_bytes": (C.c_size_t, [C.c_void_p]),
    "fdtd_save_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fdtd_load_state": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fdtd_get_step": (C.c_int64, [C.c_void_p]),
    "fdtd_set_step": (C.c_int, [C.c_void_p, C.c_int64]),
    "fdtd_get_dt": (C.c_double, [C.c_void_p]),
    "fdtd_antenna_points": (C.c_int64, [C.c_void_p, C.c_int]),
    "fdtd_sync": (C.c_int, [C.c_void_p]),
    "fdtd_set_tile": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "fdtd_step_timed": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_float), C.c_int, C.POINTER(C.c_int)]),
    "fdtd_debug_inject_fault": (C.c_int, [C.c_void_p, C.c_int]),
    "fdtd_debug_set_device": (C.c_int, [C.c_void_p, C.c_int]),
    "fdtd_set_balance": (C.c_int, [C.c_void_p, C.c_float, C.c_float]),
    "fdtd_batch_set_grid_mode": (C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    "fdtd_probe_record": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "fdtd_batch_get_grid_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "fdtd_batch_get_grid_ctas": (C.c_int, [C.c_void_p, C.c_int]),
    "fdtd_batch_autotune_bytes": (C.c_size_t, [C.c_void_p]),
    "fdtd_batch_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_size_t]),
    "fdtd_measure_fp64_rate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]),
    "fdtd_debug_vec_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "fdtd_get_balance": (C.c_int, [C.c_void_p, C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "fdtd_get_tile": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "fdtd_autotune": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fdtd_measure_balance": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fdtd_debug_tb2_order": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p]),
    "fdtd_debug_tb2_refine": (C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "fdtd_destroy_grid": (None, [C.c_void_p]),
    "fdtd_batch_required_bytes": (C.c_size_t, [C.c_int, C.c_int]),
    "fdtd_batch_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                    C.POINTER(C.c_void_p)]),
    "fdtd_batch_set_engine": (C.c_int, [C.c_void_p, C.c_int]),
    "fdtd_batch_get_engine": (C.c_int, [C.c_void_p]),
    "fdtd_batch_debug_inject_fault": (C.c_int, [C.c_void_p, C.c_int]),
    "fdtd_batch_step": (C.c_int, [C.c_void_p, C.c_int]),
    "fdtd_batch_sync": (C.c_int, [C.c_void_p]),
    "fdtd_batch_work_items": (C.c_int, [C.c_void_p]),
    "fdtd_batch_destroy": (None, [C.c_void_p]),
    "fdtd_adjoint_required_bytes": (C.c_size_t, [C.c_void_p, C.c_int64]),
    "fdtd_adjoint_create": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64, C.c_void_p, C.c_size_t,
                                      C.POINTER(C.c_void_p)]),
    "fdtd_adjoint_reset": (C.c_int, [C.c_void_p, C.c_int64]),
    "fdtd_probe_read": (C.c_int, [C.c_void_p, C.c_void_p]),
    "fdtd_adjoint_step": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "fdtd_adjoint_position": (C.c_int64, [C.c_void_p]),
    "fdtd_adjoint_get": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    "fdtd_adjoint_gradient": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "fdtd_adjoint_destroy": (None, [C.c_void_p]),
    "fdtd_fluence_noalloc_max_cells": (C.c_size_t, []),
    "fdtd_fluence_noalloc": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int]),
    "fdtd_source_coefficients": (C.c_int, [C.POINTER(fdtd_grid_desc), C.POINTER(fdtd_annulus_desc),
                                           C.c_void_p, C.c_void_p]),
    "fdtd_bessel_j": (C.c_double, [C.c_int, C.c_double]),
    "fdtd_status_string": (C.c_char_p, [C.c_int]),
    "fdtd_last_error": (C.c_char_p, []),
}


def lib():
    """Load (building first if needed) the CUDA library; raises if impossible."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def library_path() -> str:
    return _build.LIB


def check(status: int, where: str):
    if status != FDTD_OK:
        L = lib()
        raise FDTDError(status, where, L.fdtd_last_error().decode() or L.fdtd_status_string(status).decode())


# ---- thin wrappers with the C names -------------------------------------

def fdtd_grid_desc_default() -> fdtd_grid_desc:
    d = fdtd_grid_desc()
    lib().fdtd_grid_desc_default(C.byref(d))
    return d


def fdtd_required_bytes(d: fdtd_grid_desc) -> int:
    return int(lib().fdtd_required_bytes(C.byref(d)))


def fdtd_create_grid(d: fdtd_grid_desc, arena_ptr: int, nbytes: int, stream_ptr: int) -> int:
    h = C.c_void_p()
    check(lib().fdtd_create_grid(C.byref(d), C.c_void_p(arena_ptr), nbytes, C.c_void_p(stream_ptr),
                                 C.byref(h)), "fdtd_create_grid")
    return h.value


def fdtd_set_annulus_source(h: int, s: fdtd_annulus_desc):
    check(lib().fdtd_set_annulus_source(C.c_void_p(h), C.byref(s)), "fdtd_set_annulus_source")


def fdtd_step(h: int, nsteps: int):
    check(lib().fdtd_step(C.c_void_p(h), int(nsteps)), "fdtd_step")


def fdtd_fluence(h: int, dst_ptr: int, on_device: bool, reset: bool):
    check(lib().fdtd_fluence(C.c_void_p(h), C.c_void_p(dst_ptr), int(on_device), int(reset)), "fdtd_fluence")


def fdtd_fluence_noalloc(h: int, dst_ptr: int, on_device: bool, reset: bool):
    """fdtd_fluence with its staging buffer in a fixed array compiled into the
    library: for callers that cannot allocate device memory."""
    check(lib().fdtd_fluence_noalloc(C.c_void_p(h), C.c_void_p(dst_ptr), int(on_device), int(reset)),
          "fdtd_fluence_noalloc")


def measure_fp64_rate(chains: int = 8, iters: int = 20000, stream=None):
    """FP64 FMAs per second over all threads of the current device, and the
    kernel time in ms (fdtd_measure_fp64_rate)."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    st = stream if stream is not None else torch.cuda.current_stream()
    rate, ms = C.c_double(), C.c_double()
    check(lib().fdtd_measure_fp64_rate(C.c_void_p(sink.data_ptr()), C.c_void_p(st.cuda_stream), int(chains),
                                       int(iters), C.byref(rate), C.byref(ms)), "fdtd_measure_fp64_rate")
    return rate.value, ms.value


def debug_vec_norm(x, stream=None):
    """|S| from |S|^2 for a float64 CUDA tensor, by the device function of
    the FP64 fluence term (fdtd_debug_vec_norm)."""
    import torch
    x = x.contiguous()
    if x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError("debug_vec_norm takes a float64 CUDA tensor")
    out = torch.empty_like(x)
    st = stream if stream is not None else torch.cuda.current_stream()
    check(lib().fdtd_debug_vec_norm(C.c_void_p(x.data_ptr()), C.c_void_p(out.data_ptr()), x.numel(),
                                    C.c_void_p(st.cuda_stream)), "fdtd_debug_vec_norm")
    return out


def fdtd_fluence_noalloc_max_cells() -> int:
    return int(lib().fdtd_fluence_noalloc_max_cells())


def fdtd_get_field(h: int, comp: int, dst_ptr: int, on_device: bool):
    check(lib().fdtd_get_field(C.c_void_p(h), comp, C.c_void_p(dst_ptr), int(on_device)), "fdtd_get_field")


def fdtd_set_field(h: int, comp: int, src_ptr: int, on_device: bool):
    check(lib().fdtd_set_field(C.c_void_p(h), comp, C.c_void_p(src_ptr), int(on_device)), "fdtd_set_field")


def fdtd_bessel_j(n: int, x: float) -> float:
    return float(lib().fdtd_bessel_j(int(n), float(x)))


def make_grid_desc(nx, ny, nz, npml, dx, dy, dz, courant=0.95, precision="f32", fluence=True,
                   dt=0.0, z_walls=False, npml_z=0, **pml) -> fdtd_grid_desc:
    d = fdtd_grid_desc_default()
    d.nx, d.ny, d.nz, d.npml = nx, ny, nz, npml
    d.z_boundary = FDTD_Z_WALLS if z_walls else FDTD_Z_PERIODIC
    d.npml_z = npml_z
    d.dx, d.dy, d.dz = dx, dy, dz
    d.courant, d.dt = courant, dt
    d.precision = FDTD_F64 if precision in ("f64", "float64", "double") else FDTD_F32
    d.fluence = 1 if fluence else 0
    for k, v in pml.items():
        setattr(d, k, v)
    return d


def make_annulus_desc(m=0, theta=math.radians(20.0), pol="y", mode="TE", E0=1.0, r_center=12.0,
                      thickness=1.0, envelope="cw", ramp=10.0, T=0.0, T0=0.0, inject="all",
                      w_amp=None, w_phase=None):
    s = fdtd_annulus_desc()
    s.m, s.theta, s.pol, s.mode, s.E0 = m, theta, POL[pol], MODE[mode], E0
    s.r_center, s.thickness = r_center, thickness
    s.envelope, s.ramp, s.T, s.T0, s.inject = ENV[envelope], ramp, T, T0, INJ[inject]
    keep = []
    dp = C.POINTER(C.c_double)
    for name, arr in (("w_amp", w_amp), ("w_phase", w_phase)):
        if arr is None:
            setattr(s, name, dp())
        else:
            a = np.ascontiguousarray(arr, dtype=np.float64)
            keep.append(a)
            setattr(s, name, a.ctypes.data_as(dp))
    return s, keep


def make_wall_desc(theta=math.radians(25.0), w0=7.5, E0=1.0, envelope="cw", ramp=10.0, T=0.0, T0=0.0,
                   plane=1) -> fdtd_wall_desc:
    w = fdtd_wall_desc()
    w.theta, w.w0, w.E0, w.envelope = theta, w0, E0, ENV[envelope]
    w.ramp, w.T, w.T0, w.plane = ramp, T, T0, plane
    return w


def wall_coefficients(d: fdtd_grid_desc, w: fdtd_wall_desc):
    """Host-only FP64 precompute of the wall source: complex [ny, nx]."""
    out = np.zeros((d.ny, d.nx, 2))
    check(lib().fdtd_wall_coefficients(C.byref(d), C.byref(w), out.ctypes.data), "fdtd_wall_coefficients")
    return out[..., 0] + 1j * out[..., 1]


def tb2_order(t: int, u: int, nz: int, slots: int, order: int):
    """Host logic of tile variant 7 (fdtd_debug_tb2_order): (D, window at
    each flattened position)."""
    out = np.zeros(t * u, np.int32)
    D = lib().fdtd_debug_tb2_order(int(t), int(u), int(nz), int(slots), int(order), out.ctypes.data)
    if D < 0:
        raise FDTDError(FDTD_EINVAL, "fdtd_debug_tb2_order", "invalid argument")
    return D, out


def tb2_refine(starts, cycles, step: float = 1.0):
    """One refinement step of the variant-7 ranges on host data
    (fdtd_debug_tb2_refine): the new starts."""
    st = np.ascontiguousarray(starts, np.int64)
    cy = np.ascontiguousarray(cycles, np.uint64)
    if cy.size + 1 != st.size:
        raise ValueError("cycles needs one entry per range")
    out = np.zeros_like(st)
    check(lib().fdtd_debug_tb2_refine(int(cy.size), st.ctypes.data, cy.ctypes.data, float(step), out.ctypes.data),
          "fdtd_debug_tb2_refine")
    return out


def source_coefficients(d: fdtd_grid_desc, s: fdtd_annulus_desc):
    """Host-only FP64 precompute: (coef[6, ny, nx] complex, mask[ny, nx] uint8)."""
    out = np.zeros((6, d.ny, d.nx, 2))
    mask = np.zeros((d.ny, d.nx), np.uint8)
    check(lib().fdtd_source_coefficients(C.byref(d), C.byref(s), out.ctypes.data, mask.ctypes.data),
          "fdtd_source_coefficients")
    return out[..., 0] + 1j * out[..., 1], mask


# ---- torch-owned grid ----------------------------------------------------

class Grid:
    """A grid living in a torch-allocated device arena on the current stream."""

    def __init__(self, desc: fdtd_grid_desc, device=None, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libfdtd_gb300 needs a CUDA device; there is no CPU fallback")
        self.torch = torch
        self.desc = desc
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        nbytes = fdtd_required_bytes(desc)
        if nbytes == 0:
            check(FDTD_EINVAL, "fdtd_required_bytes")
        self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.arena.data_ptr()
        off = (-base) % 256
        self._arena_ptr = base + off
        with torch.cuda.device(self.device):
            self.handle = fdtd_create_grid(desc, self._arena_ptr, nbytes, self.stream.cuda_stream)
        self.dtype = torch.float64 if desc.precision == FDTD_F64 else torch.float32
        self.shape = (desc.nz, desc.ny, desc.nx)
        self._keep = None

    # source
    def set_source(self, **kw):
        s, keep = make_annulus_desc(**kw)
        self._keep = keep
        fdtd_set_annulus_source(self.handle, s)

    def clear_source(self):
        check(lib().fdtd_clear_source(C.c_void_p(self.handle)), "fdtd_clear_source")

    def set_wall_source(self, **kw):
        """The Bessel-Gauss wall sheet (fdtd_set_wall_source); keywords of make_wall_desc."""
        w = make_wall_desc(**kw)
        check(lib().fdtd_set_wall_source(C.c_void_p(self.handle), C.byref(w)), "fdtd_set_wall_source")

    def clear_wall_source(self):
        check(lib().fdtd_set_wall_source(C.c_void_p(self.handle), None), "fdtd_set_wall_source")

    def step(self, n: int = 1):
        fdtd_step(self.handle, n)

    def step_timed(self, n: int) -> list[float]:
        """Step n times, timing each kernel of a step with CUDA events:
        milliseconds per kernel of a step, summed over the n steps."""
        ms = (C.c_float * 4)()
        npass = C.c_int()
        check(lib().fdtd_step_timed(C.c_void_p(self.handle), int(n), ms, 4, C.byref(npass)), "fdtd_step_timed")
        return [float(ms[p]) for p in range(npass.value)]

    def inject_fault(self, kind: int = 1):
        """Test hook: the next step of a TMA variant withholds one bulk copy,
        so that its bounded device wait expires (fdtd_debug_inject_fault)."""
        check(lib().fdtd_debug_inject_fault(C.c_void_p(self.handle), int(kind)), "fdtd_debug_inject_fault")

    def debug_set_device(self, device: int):
        """Test hook: record `device` as the grid's device (fdtd_debug_set_device)."""
        check(lib().fdtd_debug_set_device(C.c_void_p(self.handle), int(device)), "fdtd_debug_set_device")

    def set_tile(self, variant: int, ty: int, lz: int):
        check(lib().fdtd_set_tile(C.c_void_p(self.handle), int(variant), int(ty), int(lz)), "fdtd_set_tile")

    def set_balance(self, w_shell: float, w_antenna: float):
        """Work-split weights of tile variant 7 (fdtd_set_balance)."""
        check(lib().fdtd_set_balance(C.c_void_p(self.handle), float(w_shell), float(w_antenna)), "fdtd_set_balance")

    def balance(self):
        ws, wa = C.c_float(), C.c_float()
        check(lib().fdtd_get_balance(C.c_void_p(self.handle), C.byref(ws), C.byref(wa)), "fdtd_get_balance")
        return ws.value, wa.value

    def measure_balance(self):
        """Balance the variant-7 ranges on per-window costs measured in one
        launch (fdtd_measure_balance; the state is saved and restored)."""
        scratch = self.torch.empty(self.state_bytes(), dtype=self.torch.uint8, device=self.device)
        check(lib().fdtd_measure_balance(C.c_void_p(self.handle), C.c_void_p(scratch.data_ptr())),
              "fdtd_measure_balance")
        del scratch

    def tile(self):
        v, ty, lz = C.c_int(), C.c_int(), C.c_int()
        check(lib().fdtd_get_tile(C.c_void_p(self.handle), C.byref(v), C.byref(ty), C.byref(lz)),
              "fdtd_get_tile")
        return v.value, ty.value, lz.value

    def autotune(self, steps: int = 5):
        scratch = self.torch.empty(self.state_bytes(), dtype=self.torch.uint8, device=self.device)
        check(lib().fdtd_autotune(C.c_void_p(self.handle), int(steps), C.c_void_p(scratch.data_ptr())),
              "fdtd_autotune")
        del scratch
        return self.tile()

    def sync(self):
        check(lib().fdtd_sync(C.c_void_p(self.handle)), "fdtd_sync")

    @property
    def n(self) -> int:
        return int(lib().fdtd_get_step(C.c_void_p(self.handle)))

    @property
    def dt(self) -> float:
        return float(lib().fdtd_get_dt(C.c_void_p(self.handle)))

    def antenna_points(self, comp: int) -> int:
        return int(lib().fdtd_antenna_points(C.c_void_p(self.handle), comp))

    def field(self, comp: int):
        out = self.torch.empty(self.shape, dtype=self.dtype, device=self.device)
        fdtd_get_field(self.handle, comp, out.data_ptr(), True)
        return out

    def fields(self):
        return [self.field(c) for c in range(6)]

    def set_field(self, comp: int, values):
        t = self.torch.as_tensor(values, dtype=self.dtype).to(self.device).contiguous()
        assert tuple(t.shape) == self.shape
        fdtd_set_field(self.handle, comp, t.data_ptr(), True)

    def fluence(self, reset: bool = False):
        out = self.torch.empty(self.shape, dtype=self.torch.float64, device=self.device)
        fdtd_fluence(self.handle, out.data_ptr(), True, reset)
        return out

    def state_bytes(self) -> int:
        return int(lib().fdtd_state_bytes(C.c_void_p(self.handle)))

    def save_state(self, buf=None):
        if buf is None:
            buf = self.torch.empty(self.state_bytes(), dtype=self.torch.uint8, device=self.device)
        check(lib().fdtd_save_state(C.c_void_p(self.handle), C.c_void_p(buf.data_ptr())), "fdtd_save_state")
        return buf

    def load_state(self, buf):
        check(lib().fdtd_load_state(C.c_void_p(self.handle), C.c_void_p(buf.data_ptr())), "fdtd_load_state")

    def close(self):
        if getattr(self, "handle", None):
            lib().fdtd_destroy_grid(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


BATCH_PERSISTENT, BATCH_CELL, BATCH_PERSISTENT_CELL = 0, 1, 2
BATCH_MODE_CELL4, BATCH_MODE_CELL8, BATCH_MODE_CELL16, BATCH_MODE_TWO_STEP = 0, 1, 2, 3


class Batch:
    """Several Grid objects advanced together (fdtd_batch_*): engine
    BATCH_CELL (a 64-step CUDA graph with one branch per grid, each grid in
    its own mode: cell passes on 32 x 4 / 8 / 16 blocks or the two-step
    kernel; the default) or BATCH_PERSISTENT_CELL (one cooperative launch
    per 64 steps)."""

    def __init__(self, grids, engine: int | None = None):
        import torch
        self.torch = torch
        self.grids = list(grids)
        g0 = self.grids[0]
        n = len(self.grids)
        nbytes = int(lib().fdtd_batch_required_bytes(n, g0.desc.precision))
        if nbytes == 0:
            check(FDTD_EINVAL, "fdtd_batch_required_bytes")
        self.table = torch.empty(nbytes + 256, dtype=torch.uint8, device=g0.device)
        ptr = self.table.data_ptr()
        ptr += (-ptr) % 256
        arr = (C.c_void_p * n)(*[g.handle for g in self.grids])
        h = C.c_void_p()
        check(lib().fdtd_batch_create(arr, n, C.c_void_p(ptr), nbytes, C.c_void_p(g0.stream.cuda_stream),
                                      C.byref(h)), "fdtd_batch_create")
        self.handle = h.value
        if engine is not None:
            self.set_engine(engine)

    def set_engine(self, engine: int):
        check(lib().fdtd_batch_set_engine(C.c_void_p(self.handle), int(engine)), "fdtd_batch_set_engine")

    @property
    def engine(self) -> int:
        return int(lib().fdtd_batch_get_engine(C.c_void_p(self.handle)))

    def set_grid_mode(self, q: int, mode: int):
        """Mode of grid q in the graph engine (fdtd_batch_set_grid_mode)."""
        check(lib().fdtd_batch_set_grid_mode(C.c_void_p(self.handle), int(q), int(mode)), "fdtd_batch_set_grid_mode")

    def grid_mode(self, q: int) -> int:
        return int(lib().fdtd_batch_get_grid_mode(C.c_void_p(self.handle), int(q)))

    def grid_ctas(self, q: int) -> int:
        return int(lib().fdtd_batch_get_grid_ctas(C.c_void_p(self.handle), int(q)))

    def autotune(self, steps: int = 8):
        """fdtd_batch_autotune: each grid's mode, then the engine; the grids'
        states are restored.  Returns (engine, [mode of each grid])."""
        nbytes = int(lib().fdtd_batch_autotune_bytes(C.c_void_p(self.handle)))
        scratch = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.grids[0].device)
        check(lib().fdtd_batch_autotune(C.c_void_p(self.handle), int(steps), C.c_void_p(scratch.data_ptr()),
                                        C.c_size_t(nbytes)), "fdtd_batch_autotune")
        del scratch
        return self.engine, [self.grid_mode(q) for q in range(len(self.grids))]

    def inject_fault(self, kind: int = 1):
        """Test hook: the next persistent cell launch loses one CTA, so that
        the grid barrier's bounded wait expires (fdtd_batch_debug_inject_fault)."""
        check(lib().fdtd_batch_debug_inject_fault(C.c_void_p(self.handle), int(kind)),
              "fdtd_batch_debug_inject_fault")

    def step(self, n: int = 1):
        check(lib().fdtd_batch_step(C.c_void_p(self.handle), int(n)), "fdtd_batch_step")

    def sync(self):
        check(lib().fdtd_batch_sync(C.c_void_p(self.handle)), "fdtd_batch_sync")

    @property
    def work_items(self) -> int:
        return int(lib().fdtd_batch_work_items(C.c_void_p(self.handle)))

    def close(self):
        if getattr(self, "handle", None):
            lib().fdtd_batch_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Adjoint:
    """Reverse-time adjoint of a Grid (fdtd_adjoint_*): probes of one E
    component, loss-gradient injection, and dL/dw per antenna column."""

    def __init__(self, grid: Grid, component: int, probe_cells):
        import torch
        self.torch = torch
        self.grid = grid
        cells = np.ascontiguousarray(np.asarray(probe_cells, dtype=np.int64).ravel())
        self.n_probes = int(cells.size)
        nbytes = int(lib().fdtd_adjoint_required_bytes(C.c_void_p(grid.handle), self.n_probes))
        if nbytes == 0:
            check(FDTD_EINVAL, "fdtd_adjoint_required_bytes")
        self.arena = torch.empty(nbytes + 256, dtype=torch.uint8, device=grid.device)
        ptr = self.arena.data_ptr()
        ptr += (-ptr) % 256
        h = C.c_void_p()
        check(lib().fdtd_adjoint_create(C.c_void_p(grid.handle), int(component), cells.ctypes.data,
                                        self.n_probes, C.c_void_p(ptr), nbytes, C.byref(h)), "fdtd_adjoint_create")
        self.handle = h.value
        self.component = component

    def probe_read(self, out=None):
        if out is None:
            out = self.torch.empty(self.n_probes, dtype=self.grid.dtype, device=self.grid.device)
        check(lib().fdtd_probe_read(C.c_void_p(self.handle), C.c_void_p(out.data_ptr())), "fdtd_probe_read")
        return out

    def record(self, nsteps: int):
        """Step the grid nsteps times, recording the probes after each step
        (fdtd_probe_record): a (nsteps, n_probes) device tensor."""
        out = self.torch.empty((nsteps, self.n_probes), dtype=self.grid.dtype, device=self.grid.device)
        if nsteps > 0:
            check(lib().fdtd_probe_record(C.c_void_p(self.handle), int(nsteps), C.c_void_p(out.data_ptr()),
                                          self.n_probes), "fdtd_probe_record")
        return out

    def reset(self, n_end: int):
        check(lib().fdtd_adjoint_reset(C.c_void_p(self.handle), int(n_end)), "fdtd_adjoint_reset")

    def step(self, nsteps: int, dLdE=None):
        """nsteps reverse steps; dLdE (nsteps, n_probes) device tensor of the
        grid's precision, row r = dL/dE at the (r+1)-th latest state, or None."""
        if dLdE is None:
            check(lib().fdtd_adjoint_step(C.c_void_p(self.handle), int(nsteps), None, 0), "fdtd_adjoint_step")
        else:
            t = dLdE.to(self.grid.dtype).contiguous()
            assert t.shape[0] >= nsteps and t.shape[1] == self.n_probes
            check(lib().fdtd_adjoint_step(C.c_void_p(self.handle), int(nsteps), C.c_void_p(t.data_ptr()),
                                          self.n_probes), "fdtd_adjoint_step")
            self._keep = t

    @property
    def position(self) -> int:
        return int(lib().fdtd_adjoint_position(C.c_void_p(self.handle)))

    def field(self, comp: int):
        out = self.torch.empty(self.grid.shape, dtype=self.grid.dtype, device=self.grid.device)
        check(lib().fdtd_adjoint_get(C.c_void_p(self.handle), int(comp), C.c_void_p(out.data_ptr())),
              "fdtd_adjoint_get")
        return out

    def gradient(self):
        d = self.grid.desc
        ga = self.torch.empty((d.ny, d.nx), dtype=self.torch.float64, device=self.grid.device)
        gp = self.torch.empty((d.ny, d.nx), dtype=self.torch.float64, device=self.grid.device)
        check(lib().fdtd_adjoint_gradient(C.c_void_p(self.handle), C.c_void_p(ga.data_ptr()),
                                          C.c_void_p(gp.data_ptr()), 1), "fdtd_adjoint_gradient")
        return ga, gp

    def close(self):
        if getattr(self, "handle", None):
            lib().fdtd_adjoint_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
