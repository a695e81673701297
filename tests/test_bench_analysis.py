"""Host-side analysis of the long-horizon comparison in bench.py (no GPU):
the lift period from upward mean crossings, means and amplitudes, and the
first local maximum used to align phases (Sec. 3.4)."""
import math

import bench


def test_series_summary_of_a_sinusoid():
    dt, period = 0.005, 0.31
    t = [i * dt for i in range(200)]
    lift = [0.2 + 0.05 * math.sin(2 * math.pi * x / period + 0.4) for x in t]
    drag = [3.0 + 0.01 * math.cos(4 * math.pi * x / period) for x in t]
    s = bench.series_summary(t, drag, lift)
    assert abs(s["lift_period"] - period) < 1e-3 * period
    assert abs(s["lift_amp"] - 0.05) < 1e-3 and abs(s["lift_mean"] - 0.2) < 5e-3
    assert abs(s["drag_mean"] - 3.0) < 1e-3 and abs(s["drag_amp"] - 0.01) < 1e-4


def test_steady_series_has_no_period():
    t = [i * 0.005 for i in range(50)]
    s = bench.series_summary(t, [2.5] * 50, [0.0] * 50)
    assert s["lift_period"] is None and s["lift_amp"] == 0.0


def test_first_max_and_phase_shift():
    dt, period = 0.005, 0.2
    t = [i * dt for i in range(120)]
    a = [math.sin(2 * math.pi * x / period) for x in t]
    b = [math.sin(2 * math.pi * (x - 7 * dt) / period) for x in t]   # lags a by 7 steps
    assert bench.first_max(a) == 10          # sin peaks at t = period / 4 = 10 steps
    assert bench.first_max(b) - bench.first_max(a) == 7
    assert bench.first_max([1.0, 0.5, 0.2]) is None
