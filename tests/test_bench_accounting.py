"""Host-side checks of bench.py's roofline accounting (no GPU): the
algorithmic bytes per cell of each kernel follow from the arrays each pass
must read and write, and the per-kernel achieved bandwidth is those bytes
over the measured duration."""
import pytest

import bench
from paper_2102_12978_gb300 import workloads as W


def test_psi_per_cell_counts_every_shell():
    w = W.config2()                                   # 256 x 256 x 128, 16-cell CPML on x and y
    assert bench.psi_per_cell(w) == pytest.approx(4 * 32 / 256 + 4 * 32 / 256)   # = 1.0
    b = W.bessel_gauss()                              # 411 x 411 x 738, 16 cells on all six faces
    assert bench.psi_per_cell(b) == pytest.approx(4 * 32 / 411 * 2 + 4 * 32 / 738)


def test_pass_bytes_of_the_256_workload():
    """FP32: the H pass moves E^n, H^{n-1/2} in and H^{n+1/2} out (36 B) plus
    its psi (4 B on average); the E pass E^n, H^{n+1/2}, H^{n-1/2} in and
    E^{n+1} out (48 B), the 8-byte fluence in and out (16 B) and its psi
    (4 B); one pass moves 12 words, the fluence and all psi twice: 72 B."""
    w = W.config2()
    assert bench.pass_bytes_per_cell(w, 5, 4) == [("yee_h_cell", 40.0), ("yee_e_cell", 68.0)]
    assert bench.pass_bytes_per_cell(w, 1, 4) == [("yee_step_tma", 72.0)]
    assert bench.algorithmic_bytes_per_cell(w, 4) == 72.0
    # FP64: each cell pass is timed with its antenna pass
    assert bench.pass_bytes_per_cell(w, 5, 8) == [("yee_h_cell + antenna_add", 80.0),
                                                  ("yee_e_cell + antenna_add", 120.0)]


def test_bessel_gauss_pass_bytes_include_the_z_shells():
    b = W.bessel_gauss()
    (h, hb), (e, eb) = bench.pass_bytes_per_cell(b, 5, 4)
    assert hb == pytest.approx(36 + 4 * bench.psi_per_cell(b))
    assert eb == pytest.approx(64 + 4 * bench.psi_per_cell(b))
    assert hb == pytest.approx(39.185, abs=1e-3) and eb == pytest.approx(67.185, abs=1e-3)


def test_kernel_roofline_is_bytes_over_time():
    w = W.config2()
    cells = w.cells
    rows, dom = bench.kernel_roofline(w, (5, 4, 1), [65.6 * 100 / 1000, 117.3 * 100 / 1000], 100, 4, 6695.0, cells)
    assert [r["kernel"] for r in rows] == ["yee_h_cell", "yee_e_cell"]
    assert dom["kernel"] == "yee_e_cell"
    assert rows[1]["achieved_gbs"] == pytest.approx(68 * cells / 117.3e-6 / 1e9, rel=1e-3)
    assert rows[1]["frac"] == pytest.approx(rows[1]["achieved_gbs"] / 6695.0, rel=1e-3)


def test_job_rate_counts_every_rank():
    assert bench.job_rate(8 * 10 ** 6, 100, 2, 1000.0) == pytest.approx(1.6)


def test_two_step_kernel_accounting():
    """Variant 7 advances two steps per launch: its algorithmic bytes per
    launch are the method's 72 B for each of the two cell-updates, a launch
    lasts the summed event time over steps / 2 launches, and a block of K steps
    takes K / 2 launches (an odd K adds one two-pass step)."""
    w = W.config2()
    cells = w.cells
    assert bench.pass_bytes_per_cell(w, 7, 4) == [("yee_tb2", 144.0)]
    rows, dom = bench.kernel_roofline(w, (7, 16, 1), [150.0], 1000, 4, 6768.4, cells)
    assert dom["ms_per_launch"] == pytest.approx(0.3)
    assert dom["achieved_gbs"] == pytest.approx(144 * cells / 0.3e-3 / 1e9, rel=1e-4)
    assert bench.launches_per_block(7, 20) == 10
    assert bench.launches_per_block(7, 21) == 12
    assert bench.launches_per_block(5, 20) == 40
    assert bench.launches_per_block(1, 20) == 20


def test_step_traffic_is_per_step():
    saved = dict(bench.TRAFFIC)
    try:
        bench.TRAFFIC.update({"yee_h_cell": 300e6, "yee_e_cell": 500e6, "yee_tb2": 1000e6})
        assert bench.step_traffic(5) == 800e6
        assert bench.step_traffic(7) == 500e6
        bench.TRAFFIC["yee_tb2"] = None
        assert bench.step_traffic(7) is None
        assert bench.step_traffic(3) is None
    finally:
        bench.TRAFFIC.clear()
        bench.TRAFFIC.update(saved)
