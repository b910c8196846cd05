"""Pins of the oracle's reverse-time adjoint: the exact transpose of its own
discrete step (dot-product identity, CPML and PEC included) and agreement of
the weight gradients with central finite differences of the forward run."""
import numpy as np
import pytest

import oracle
from paper_2102_12978_gb300 import workloads as W
from tests.cases import oracle_grid, oracle_source


def _fill_random(st, rng):
    for arr in (*st.e, *st.h, *st.psi_e, *st.psi_h):
        arr[...] = rng.standard_normal(arr.shape)


def _dot(a, b):
    return sum(float(np.sum(x * y)) for x, y in zip((*a.e, *a.h, *a.psi_e, *a.psi_h),
                                                    (*b.e, *b.h, *b.psi_e, *b.psi_h)))


@pytest.mark.parametrize("npml,steps", [(0, 1), (4, 1), (4, 3)])
def test_dot_product_identity(npml, steps):
    """<M x, y> = <x, M^T y> for random full states (fields and psi)."""
    g = oracle.Grid(18, 16, 6, npml, 0.06, 0.055, 0.07, courant=0.9)
    rng = W.rng(11)
    x = oracle.State(g, fluence=False)
    y = oracle.State(g, fluence=False)
    _fill_random(x, rng)
    _fill_random(y, rng)
    mx = x.copy()
    oracle.run(g, None, mx, steps)
    mty = y.copy()
    for n in reversed(range(steps)):
        oracle.adjoint_step(g, None, mty, n)
    lhs, rhs = _dot(mx, y), _dot(x, mty)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + abs(rhs)), (lhs, rhs)


def _probe_loss_setup(seed=5):
    w = W.small(nx=30, ny=28, nz=6, npml=4, r_center=7.0, steps=25, ramp=0.5, theta_deg=25.0)
    g = oracle_grid(w)
    rng = W.rng(seed)
    amp = 1.0 + 0.2 * rng.standard_normal((w.ny, w.nx))
    ph = 0.3 * rng.standard_normal((w.ny, w.nx))
    probes = rng.integers(0, w.nx * w.ny * w.nz, size=40)
    return w, g, amp, ph, probes


def _forward_epol(w, g, amp, ph, window):
    st = oracle.State(g, fluence=False)
    src = oracle_source(w, w_amp=amp, w_phase=ph)
    oracle.run(g, src, st, w.steps - window)
    rows = []
    for _ in range(window):
        oracle.run(g, src, st, 1)
        rows.append(st.e[1].ravel().copy())
    return rows


def test_gradient_matches_central_differences():
    """L = sum over a window of sum_p E_y(p)^2 at random probe cells; the
    adjoint's dL/dw_amp and dL/dw_phase against central differences."""
    w, g, amp, ph, probes = _probe_loss_setup()
    window = 6

    def loss(a, p):
        rows = _forward_epol(w, g, a, p, window)
        return sum(float(np.sum(r[probes] ** 2)) for r in rows)

    # adjoint: the reverse run injects dL/dE^n = 2 E^n at the probes
    rows = _forward_epol(w, g, amp, ph, window)
    src = oracle_source(w, w_amp=amp, w_phase=ph)
    adj = oracle.State(g, fluence=False)
    ga = np.zeros((w.ny, w.nx)); gp = np.zeros((w.ny, w.nx))
    for n in reversed(range(w.steps)):
        r = n - (w.steps - window)            # E^{n+1} is row r of the window
        if 0 <= r < window:
            flat = adj.e[1].reshape(-1)
            np.add.at(flat, probes, 2.0 * rows[r][probes])
        oracle.adjoint_step(g, src, adj, n, ga, gp)
    # the antenna columns with the largest gradient
    cols = np.argsort(-np.abs(ga).ravel())[:3]
    h = 1e-6
    for c in cols:
        j, i = divmod(int(c), w.nx)
        for which, grad in (("amp", ga), ("phase", gp)):
            a1, a2 = amp.copy(), amp.copy()
            p1, p2 = ph.copy(), ph.copy()
            if which == "amp":
                a1[j, i] += h; a2[j, i] -= h
            else:
                p1[j, i] += h; p2[j, i] -= h
            fd = (loss(a1, p1) - loss(a2, p2)) / (2 * h)
            assert abs(fd - grad[j, i]) <= 1e-6 * max(1.0, abs(fd)), (which, fd, grad[j, i])
