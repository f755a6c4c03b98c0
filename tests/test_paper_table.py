"""The paper's only printed numbers (Table 1) and the reading of its columns.

'Speed ratio' is realtime factor: (100 IPPs x 10 ms) / time; 'speedup' is the CPU time
over the row's time.  These readings turn the table into the spectra/s context figures
quoted beside the benchmark.
"""
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    with open(os.path.join(HERE, "golden", "table1_paper_timings.json")) as fh:
        return json.load(fh)


def test_speed_ratio_is_realtime_factor():
    t = _table()
    for row in t["rows"]:
        ratio = 100 * t["realtime_ipp_seconds"] / row["time_s"]
        assert abs(ratio - row["speed_ratio"]) <= 0.0015, row


def test_speedup_is_cpu_time_over_time():
    t = _table()
    cpu = t["rows"][0]["time_s"]
    for row in t["rows"]:
        assert abs(cpu / row["time_s"] - row["speedup"]) <= 0.006, row


def test_derived_spectra_per_second():
    # 100 IPPs x 4096 gates transforms per run
    t = _table()
    best = max(100 * 4096 / r["time_s"] for r in t["rows"])
    assert 275_000 < best < 275_500
