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


def _summary(errs):
    return {k: {"vel_l2_err_mean": v} for k, v in errs.items()}


def test_equal_error_interpolates_between_bracketing_points():
    """MG(L+1)'s time at DNN-MG's error: log(time) linear in log(error)
    between the two sweep points around the target error (Sec. 3.3's
    comparison of time per step at equal accuracy)."""
    K = 10
    errs = {"dnnmg": 1e-4, "a": 1e-8, "b": 1e-5, "c": 1e-3}
    times = {"dnnmg": 50.0, "a": 200.0, "b": 100.0, "c": 40.0}   # summed over K steps
    eq = bench.equal_error(times, _summary(errs), K, ["a", "b", "c"])
    assert eq["bracketed"] and eq["between"] == ["b", "c"]
    # 1e-4 is halfway between 1e-5 and 1e-3 in log scale: sqrt(10 * 4) ms
    assert abs(eq["mg_fine_ms_at_equal_error"] - math.sqrt(10.0 * 4.0)) < 1e-12
    assert abs(eq["speedup_vs_mg_fine"] - math.sqrt(40.0) / 5.0) < 1e-12
    assert [p["run"] for p in eq["sweep"]] == ["a", "b", "c"]


def test_equal_error_unbracketed_gives_an_upper_bound():
    K = 4
    errs = {"dnnmg": 1e-2, "a": 1e-8, "b": 1e-5}
    times = {"dnnmg": 20.0, "a": 80.0, "b": 24.0}
    eq = bench.equal_error(times, _summary(errs), K, ["a", "b"])
    assert not eq["bracketed"] and eq["between"] == ["b", None]
    assert eq["mg_fine_ms_at_equal_error"] == 6.0 and eq["speedup_vs_mg_fine"] == 6.0 / 5.0


def test_equal_error_unbracketed_takes_the_fastest_accurate_point():
    """When every sweep point is more accurate than the target, the bound is
    the fastest of them, not necessarily the loosest (the loosest can be the
    slower one, e.g. a one-Newton-step, one-V-cycle point)."""
    K = 2
    errs = {"dnnmg": 1e-3, "a": 1e-9, "b": 1e-5, "c": 3e-5}
    times = {"dnnmg": 6.0, "a": 18.0, "b": 3.4, "c": 4.8}
    eq = bench.equal_error(times, _summary(errs), K, ["a", "b", "c"])
    assert not eq["bracketed"] and eq["between"] == ["b", None]
    assert eq["mg_fine_ms_at_equal_error"] == 1.7
    assert abs(eq["speedup_vs_mg_fine"] - 1.7 / 3.0) < 1e-15


def test_source_hash_is_stable_and_covers_the_sources():
    h = bench.source_hash()
    assert len(h) == 16 and h == bench.source_hash()
