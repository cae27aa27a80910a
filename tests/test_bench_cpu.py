"""CPU checks of the benchmark's host-side arithmetic: the unit-trace summary
of the batched form, the clock record, and the oracle-rate extrapolation.
No GPU and no library calls."""
import os
import types

import numpy as np

import bench


def _trace(rows):
    """rows: (t0 ms, t1 ms, problem, G) -> the dict Context.batch_trace_read returns."""
    r = np.array(rows, dtype=np.float64)
    base = 1_000_000_000  # ns: stamps are absolute global-timer values
    return dict(t0=(base + r[:, 0] * 1e6).astype(np.uint64), t1=(base + r[:, 1] * 1e6).astype(np.uint64),
                problem=r[:, 2].astype(np.int64), sm=np.zeros(len(rows), dtype=np.int64),
                s0=np.zeros(len(rows), dtype=np.int64), starts=np.ones(len(rows), dtype=np.int64),
                G=r[:, 3].astype(np.int64))


def test_unit_trace_summary_finds_the_critical_unit():
    # three units run together for 2 ms, one of them for 10 ms; a fourth
    # starts at 2 ms and ends at 3 ms
    tr = _trace([(0.0, 10.0, 0, 32), (0.0, 2.0, 1, 16), (0.0, 2.0, 2, 16), (2.0, 3.0, 1, 16)])
    probs = [types.SimpleNamespace(n=5, L=10), types.SimpleNamespace(n=3, L=4),
             types.SimpleNamespace(n=4, L=6)]
    info = [dict(sweeps=500, converged=False), dict(sweeps=12, converged=True), dict(sweeps=30, converged=True)]
    s = bench.unit_trace_summary(tr, probs, info)
    assert s["units"] == 4
    assert abs(s["span_ms"] - 10.0) < 1e-9
    assert s["peak_concurrent_units"] == 3
    # full (>= 90% of the peak) only while all three ran: up to the last grid point before 2 ms
    assert 2.0 - 10.0 / 400 - 1e-9 <= s["full_until_ms"] < 2.0
    assert abs(s["tail_ms"] - (s["span_ms"] - s["full_until_ms"])) < 1e-12
    last = s["last_unit"]
    assert (last["n"], last["L"], last["converged"], last["sweeps"], last["lanes_per_start"]) == (5, 10, False, 500, 32)
    assert last["start_ms"] == 0.0 and abs(last["duration_ms"] - 10.0) < 1e-9
    assert abs(last["us_per_sweep"] - 20.0) < 1e-9


def test_unit_trace_summary_of_an_empty_trace():
    empty = {k: np.zeros(0, dtype=np.uint64 if k in ("t0", "t1") else np.int64)
             for k in ("t0", "t1", "problem", "sm", "s0", "starts", "G")}
    assert bench.unit_trace_summary(empty, [], []) is None


def test_clock_record_median_under_load_and_reasons(tmp_path):
    path = tmp_path / "clocks.csv"
    lines = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1100.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 345, 2070, 150.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",  # idle
        "garbage line",
    ]
    path.write_text("\n".join(lines) + "\n")
    c = bench.Clocks(0)
    c.path = str(path)
    c.fh = open(os.devnull, "w")
    c.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0, kill=lambda: None)
    rec = c.stop()
    assert rec["sm_mhz"] == 2070.0  # median of the loaded samples (the idle one is dropped)
    assert rec["sm_max_mhz"] == 2070.0
    assert rec["reasons"] == ["sw_power_cap"]
    assert rec["samples"] == 4


def test_clock_record_without_nvidia_smi():
    c = bench.Clocks(0)
    c.proc = None
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_oracle_rate_extrapolation():
    samples = [dict(seconds_precompute=2.0, seconds_per_sweep_all_starts=3.0),
               dict(seconds_precompute=4.0, seconds_per_sweep_all_starts=5.0)]
    g = dict(sweeps=10.0, converged=0.5)
    rate, t_inst = bench.oracle_rate(samples, g)
    assert t_inst == 0.5 * ((2.0 + 30.0) + (4.0 + 50.0))
    assert rate == 0.5 / t_inst


def test_golden_runs_summary():
    g = bench.golden_runs("brick_n12")
    assert g is not None and g["targets"] == 12 and g["seeds"] == list(range(12))
    assert 0.0 < g["converged"] <= 1.0 and g["sweeps"] > 1.0
    assert bench.golden_runs("no_such_workload") is None
