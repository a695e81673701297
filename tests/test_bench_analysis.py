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


def test_vcycle_bytes_closed_form():
    """The algorithmic bytes of one V(2,2) cycle, against the count written
    out by hand for a two-level cycle (top level 2 over the coarse level 1):
    16 colour passes of 576 B per fluid cell / 4 and 44 B per node, one
    defect of 44 B per node, the transfers (36 B per fine node, 36 B per
    coarse node), zeroing the top iterate (12 B per node), and the 891 x 891
    FP64 coarse inverse with its vector read once."""
    n2 = (16 * 4 + 1) * (4 * 4 + 1)       # 1105 nodes on level 2
    n1 = (16 * 2 + 1) * (4 * 2 + 1)       # 297 nodes on level 1
    cells2 = 64 * 16 - 4 * 16             # 960 fluid cells (the 2 x 2-cell block per level-0 cell)
    passes = 16 * (cells2 / 4 * 576 + 44 * n2)
    expect = 12 * n2 + passes + 44 * n2 + 36 * n2 + 36 * n1 + 8 * 891 * 891 + 8 * 891
    assert bench.vcycle_bytes(2) == expect
    assert bench.nnodes(2) == n2 and bench.fluid_cells(2) == cells2
    # the benchmark's figure (top level 5), quoted in the design notes
    assert bench.vcycle_bytes(5) == 265147100


def test_job_throughput_counts_every_rank():
    assert bench.job_throughput(1000.0, 10, 1) == 10.0
    assert bench.job_throughput(500.0, 10, 4) == 80.0


def test_summarize_launches_aggregates_an_ncu_launch_list(tmp_path, capsys):
    """Launches and total time per kernel (template arguments kept, the
    namespace and the parameter list dropped), units converted to us, shares
    of the total, largest first."""
    head = ["ID", "Process ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value"]
    rows = [
        ["0", "1", "void dnnmg::(anonymous namespace)::vcycle_kernel<float>(const int *)",
         "gpu__time_duration.sum", "usecond", "300"],
        ["1", "1", "void dnnmg::(anonymous namespace)::vcycle_kernel<float>(const int *)",
         "gpu__time_duration.sum", "nsecond", "100,000"],
        ["2", "1", "dnnmg::(anonymous namespace)::post_kernel(dnnmg::HostMail *)",
         "gpu__time_duration.sum", "usecond", "100"],
        ["3", "1", "dnnmg::(anonymous namespace)::post_kernel(dnnmg::HostMail *)",
         "dram__bytes_read.sum", "byte", "64"],
    ]
    p = tmp_path / "launches.csv"
    with open(p, "w", newline="") as fh:
        import csv
        w = csv.writer(fh)
        w.writerow(["==PROF== a line before the table"])
        w.writerow(head)
        w.writerows(rows)
    bench.summarize_launches(str(p))
    out = capsys.readouterr().out.splitlines()
    assert out[1].split() == ["vcycle_kernel<float>", "2", "400.0", "80.0%"]
    assert out[2].split() == ["post_kernel", "1", "100.0", "20.0%"]
