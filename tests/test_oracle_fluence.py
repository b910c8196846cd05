"""Pins of the oracle's fluence (Section 2: the time integral of |S|, S = E x H).

The oracle takes the fluence at cell centres: E averaged over the four edges
of each component around the centre, H over the two faces and over the two
half steps around t_n, and adds |E^n_c x Hbar^n_c| dt per step n = n0 .. n0+N-1
(a left Riemann sum; the reading of the fluence used throughout).

For a sinusoidal Yee eigenmode those averages have a closed form that uses no
index arithmetic: the mean of a sinusoid over two points a distance d apart
is its value at the midpoint times cos(k d / 2), and the mean over the two
half steps around t_n is the value at t_n times cos(w dt / 2).  The pins
evaluate the modes' analytic fields at the cell centres and at t_n, apply
those factors, and sum |S| dt in NumPy; the oracle, run from the discrete
modes, must agree to 1e-12.  A mistake in the averaging offsets, the time
centring, the dt factor or the range of the sum fails them, as the planted
variants below show.
"""
import math

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

N_STEPS = 50


def _grid(nx=12, ny=10, nz=16, dx=0.1, dy=0.13, dz=0.07, courant=0.9):
    return oracle.Grid(nx, ny, nz, 0, dx, dy, dz, courant=courant)


def _omega(dt, *K):
    om = math.sqrt(sum(k * k for k in K))
    return 2.0 / dt * math.asin(om * dt / 2.0), om


class Mode:
    """One closed-form Yee eigenmode of the PEC / periodic-z box.

    ``staggered(g, t_e, t_h)`` gives the discrete fields at their own Yee
    points (the oracle's initial state); ``centre(g, t, tc)`` gives E and the
    time-centred H at the cell centres ((i+1/2) dx, (j+1/2) dy, (k+1/2) dz)
    at t = n dt, already multiplied by the two-point averaging factors.
    ``tc`` scales the time-centring factor (1: the reading; planted variants
    change it)."""

    def __init__(self, kind, g):
        self.kind = kind
        if kind == "te10":
            p, r = 2, 1
            self.k = (p * np.pi / (g.nx * g.dx), 0.0, 2 * np.pi * r / (g.nz * g.dz))
        elif kind == "te01":
            q, r = 3, 2
            self.k = (0.0, q * np.pi / (g.ny * g.dy), 2 * np.pi * r / (g.nz * g.dz))
        elif kind == "tm11":
            p, q = 1, 2
            self.k = (p * np.pi / (g.nx * g.dx), q * np.pi / (g.ny * g.dy), 0.0)
        kx, ky, kz = self.k
        self.K = (2 / g.dx * np.sin(kx * g.dx / 2), 2 / g.dy * np.sin(ky * g.dy / 2),
                  2 / g.dz * np.sin(kz * g.dz / 2))
        self.w, self.Om = _omega(g.dt, *[K for K in self.K if K != 0.0])

    def staggered(self, g, t_e, t_h):
        kx, ky, kz = self.k
        Kx, Ky, Kz = self.K
        w, Om = self.w, self.Om
        k = np.arange(g.nz)[:, None, None]
        j = np.arange(g.ny)[None, :, None]
        i = np.arange(g.nx)[None, None, :]
        x0, xh = i * g.dx, (i + 0.5) * g.dx
        y0, yh = j * g.dy, (j + 0.5) * g.dy
        z0, zh = k * g.dz, (k + 0.5) * g.dz
        one = np.ones(g.shape)
        Z = np.zeros(g.shape)
        if self.kind == "te10":
            Ey = one * np.sin(kx * x0) * np.cos(kz * z0 - w * t_e)
            Hx = one * (-Kz / Om) * np.sin(kx * x0) * np.cos(kz * zh - w * t_h)
            Hz = one * (Kx / Om) * np.cos(kx * xh) * np.sin(kz * z0 - w * t_h)
            return [Z, Ey, Z.copy()], [Hx, Z.copy(), Hz]
        if self.kind == "te01":
            Ex = one * np.sin(ky * y0) * np.cos(kz * z0 - w * t_e)
            Hy = one * (Kz / Om) * np.sin(ky * y0) * np.cos(kz * zh - w * t_h)
            Hz = one * (-Ky / Om) * np.cos(ky * yh) * np.sin(kz * z0 - w * t_h)
            return [Ex, Z, Z.copy()], [Z.copy(), Hy, Hz]
        Ez = one * np.sin(kx * x0) * np.sin(ky * y0) * np.cos(w * t_e)
        Hx = one * (-Ky / Om) * np.sin(kx * x0) * np.cos(ky * yh) * np.sin(w * t_h)
        Hy = one * (Kx / Om) * np.cos(kx * xh) * np.sin(ky * y0) * np.sin(w * t_h)
        return [Z, Z.copy(), Ez], [Hx, Hy, Z.copy()]

    def centre(self, g, t, tc=1.0, shift=(0.0, 0.0, 0.0)):
        """Cell-centre E and Hbar at time t; `shift` moves the centres (in
        cells) for the planted-offset variant."""
        kx, ky, kz = self.k
        Kx, Ky, Kz = self.K
        w, Om = self.w, self.Om
        k = np.arange(g.nz)[:, None, None]
        j = np.arange(g.ny)[None, :, None]
        i = np.arange(g.nx)[None, None, :]
        xc = (i + 0.5 + shift[0]) * g.dx
        yc = (j + 0.5 + shift[1]) * g.dy
        zc = (k + 0.5 + shift[2]) * g.dz
        ax, ay, az = np.cos(kx * g.dx / 2), np.cos(ky * g.dy / 2), np.cos(kz * g.dz / 2)
        at = tc * np.cos(w * g.dt / 2)          # mean over t_n -+ dt/2
        one = np.ones(g.shape)
        Z = np.zeros(g.shape)
        if self.kind == "te10":
            # E_y averaged over x and z; H_x over x and time; H_z over z and time
            ey = one * np.sin(kx * xc) * ax * np.cos(kz * zc - w * t) * az
            hx = one * (-Kz / Om) * np.sin(kx * xc) * ax * np.cos(kz * zc - w * t) * at
            hz = one * (Kx / Om) * np.cos(kx * xc) * np.sin(kz * zc - w * t) * az * at
            return [Z, ey, Z.copy()], [hx, Z.copy(), hz]
        if self.kind == "te01":
            ex = one * np.sin(ky * yc) * ay * np.cos(kz * zc - w * t) * az
            hy = one * (Kz / Om) * np.sin(ky * yc) * ay * np.cos(kz * zc - w * t) * at
            hz = one * (-Ky / Om) * np.cos(ky * yc) * np.sin(kz * zc - w * t) * az * at
            return [ex, Z, Z.copy()], [Z.copy(), hy, hz]
        ez = one * np.sin(kx * xc) * ax * np.sin(ky * yc) * ay * np.cos(w * t)
        hx = one * (-Ky / Om) * np.sin(kx * xc) * ax * np.cos(ky * yc) * np.sin(w * t) * at
        hy = one * (Kx / Om) * np.cos(kx * xc) * np.sin(ky * yc) * ay * np.sin(w * t) * at
        return [Z, Z.copy(), ez], [hx, hy, Z.copy()]


def _closed_form_fluence(g, modes, n_steps, first=0, dt_scale=1.0, tc=1.0, shift=(0.0, 0.0, 0.0)):
    F = np.zeros(g.shape)
    for n in range(first, first + n_steps):
        E = [np.zeros(g.shape) for _ in range(3)]
        H = [np.zeros(g.shape) for _ in range(3)]
        for m in modes:
            e, h = m.centre(g, n * g.dt, tc=tc, shift=shift)
            for c in range(3):
                E[c] += e[c]
                H[c] += h[c]
        S = np.cross(np.stack(E, -1), np.stack(H, -1))
        F += np.sqrt((S * S).sum(-1)) * g.dt * dt_scale
    return F


def _oracle_fluence(g, modes, n_steps):
    st = oracle.State(g, fluence=True)
    for m in modes:
        e, h = m.staggered(g, 0.0, -0.5 * g.dt)
        for c in range(3):
            st.e[c][...] += e[c]
            st.h[c][...] += h[c]
    oracle.run(g, None, st, n_steps)
    return st.fluence


CASES = {
    "te10": ["te10"],            # E_y with H_x and H_z: the z average of H_z and E_y enters
    "te01": ["te01"],
    "tm11": ["tm11"],
    "te10+tm11": ["te10", "tm11"],   # all six components, cross terms of two frequencies
}


@pytest.mark.parametrize("case", list(CASES))
def test_oracle_fluence_matches_closed_form(case):
    g = _grid()
    modes = [Mode(k, g) for k in CASES[case]]
    F = _oracle_fluence(g, modes, N_STEPS)
    ref = _closed_form_fluence(g, modes, N_STEPS)
    assert np.abs(ref).max() > 1e-3
    err = np.abs(F - ref).max() / np.abs(ref).max()
    assert err < 1e-12, err


def test_fluence_pin_has_a_z_term():
    """TE10 travels along z: its centre S_z = -E_y H_x is nonzero and the
    fluence depends on the z average of E_y and H_z."""
    g = _grid()
    m = Mode("te10", g)
    e, h = m.centre(g, 0.3 * g.dt)
    sz = e[0] * h[1] - e[1] * h[0]
    assert np.abs(sz).max() > 0.1 * np.abs(e[1]).max() * np.abs(h[0]).max()
    assert abs(np.cos(m.k[2] * g.dz / 2) - 1.0) > 1e-3   # the z averaging factor matters


@pytest.mark.parametrize("plant", ["half_dt", "no_time_centring", "sum_from_1", "offset_x", "offset_z"])
def test_fluence_pin_detects_planted_mistakes(plant):
    """Each plausible misreading of the fluence, planted in the closed form,
    moves it far beyond the 1e-12 bound of the pin."""
    g = _grid()
    modes = [Mode("te10", g), Mode("tm11", g)]
    F = _oracle_fluence(g, modes, N_STEPS)
    kw = {
        "half_dt": dict(dt_scale=0.5),
        "no_time_centring": dict(tc=1.0 / np.cos(modes[0].w * g.dt / 2)),
        "sum_from_1": dict(first=1),
        "offset_x": dict(shift=(0.5, 0.0, 0.0)),
        "offset_z": dict(shift=(0.0, 0.0, 0.5)),
    }[plant]
    wrong = _closed_form_fluence(g, modes, N_STEPS, **kw)
    err = np.abs(F - wrong).max() / np.abs(F).max()
    assert err > 1e-6, (plant, err)
