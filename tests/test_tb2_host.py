"""Host logic of tile variant 7 (the two-step kernel), on the CPU through the
C ABI's test hooks: the interleaved window order is a bijection that puts
x-neighbouring windows the chosen stride apart, and one refinement step of
the CTAs' ranges moves each boundary to where the measured time, spread
evenly over each CTA's items, splits equally.  No kernel is launched here."""
import numpy as np
import pytest

from paper_2102_12978_gb300 import fdtd


@pytest.mark.parametrize("t,u,nz,slots", [(9, 21, 128, 152), (8, 19, 128, 152), (3, 2, 5, 152), (20, 7, 64, 152),
                                          (73, 171, 503, 152), (1, 1, 1, 1), (5, 33, 9, 40)])
def test_interleaved_order_is_a_bijection_with_x_neighbours_d_apart(t, u, nz, slots):
    D, order = fdtd.tb2_order(t, u, nz, slots, 2)
    assert 1 <= D <= min(16, u)
    assert sorted(order.tolist()) == list(range(t * u))
    pos = np.empty(t * u, np.int64)
    pos[order] = np.arange(t * u)
    for wy in range(u):
        rows = min(D, u - (wy // D) * D)   # rows of this window row's group
        for wx in range(t - 1):
            assert pos[wy * t + wx + 1] - pos[wy * t + wx] == rows
    # the stride brings D windows of planes closest to a whole number of CTA shares
    share = t * u * nz / slots
    dist = lambda d: min((nz * d) % share, share - (nz * d) % share)
    assert all(dist(D) <= dist(d) + 1e-9 for d in range(1, min(16, u) + 1))


@pytest.mark.parametrize("t,u", [(9, 21), (4, 3)])
def test_row_by_row_order_is_the_identity(t, u):
    D, order = fdtd.tb2_order(t, u, 128, 152, 1)
    assert D == 1 and order.tolist() == list(range(t * u))


def test_refine_step_moves_the_boundary_to_the_equal_time_split():
    # CTA 0 took 200 cycles for items [0, 100), CTA 1 100 cycles for [100, 200):
    # half of the 300 cycles lie at 150 / 200 of CTA 0's items
    assert fdtd.tb2_refine([0, 100, 200], [200, 100]).tolist() == [0, 75, 200]
    # damped: half of the way
    assert fdtd.tb2_refine([0, 100, 200], [200, 100], 0.5).tolist() == [0, 88, 200]


def test_refine_step_skips_empty_ranges_and_keeps_the_ends():
    out = fdtd.tb2_refine([0, 0, 50, 50, 100], [7, 100, 3, 300]).tolist()
    assert out[0] == 0 and out[-1] == 100
    assert all(a <= b for a, b in zip(out, out[1:]))
    # 400 cycles: CTA 1 (items 0-50) carries 100 of them, CTA 3 (50-100) 300
    assert out[1:4] == [50, 67, 83]


def test_refine_of_equal_times_changes_nothing():
    s = [0, 13, 40, 41, 90, 128]
    for step in (1.0, 0.75):
        assert fdtd.tb2_refine(s, [1000, 1000, 1000, 1000, 1000], step).tolist() == s
    # cycles proportional to the items: the equal split lies at equal item counts
    assert fdtd.tb2_refine(s, [13, 27, 1, 49, 38]).tolist() == [0, 26, 51, 77, 102, 128]


def test_refine_rejects_bad_input():
    with pytest.raises(fdtd.FDTDError):
        fdtd.tb2_refine([1, 2, 3], [1, 1])        # starts[0] != 0
    with pytest.raises(fdtd.FDTDError):
        fdtd.tb2_refine([0, 5, 3], [1, 1])        # decreasing
    with pytest.raises(fdtd.FDTDError):
        fdtd.tb2_refine([0, 5, 9], [1, 1], 0.0)   # step outside (0, 1]
