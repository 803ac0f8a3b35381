"""bench.py's host-side helpers without a GPU: the clock sampler's parsing of
nvidia-smi's CSV (median SM clock, the maximum, and which throttle reasons were
active at any sample) and its behaviour when nvidia-smi is missing."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _sampler_with(tmp_path, text):
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "clocks.csv")
    with open(s.path, "w") as fh:
        fh.write(text)
    s.proc = object()       # as if nvidia-smi had been started
    return s


def test_clock_summary_reports_median_max_and_active_reasons(tmp_path):
    rows = [
        "0, 2032, 2032, 812.50, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2032, 1098.10, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2032, 2032, 905.00, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
        "0, [N/A], 2032, 900.00, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = _sampler_with(tmp_path, "\n".join(rows) + "\n")
    out = s.summary()
    assert out["sm_mhz"] == 2032.0 and out["sm_max_mhz"] == 2032.0 and out["samples"] == 3
    assert out["power_w_max"] == 1098.1 and out["reasons"] == ["sw_power_cap"]


def test_clock_summary_flags_slowdowns(tmp_path):
    rows = [
        "0, 1200, 2032, 500.00, 0x8, Active, Not Active, Not Active, Not Active",
        "0, 1100, 2032, 480.00, 0x40, Not Active, Active, Active, Not Active",
    ]
    out = _sampler_with(tmp_path, "\n".join(rows) + "\n").summary()
    assert out["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert out["sm_mhz"] == 1150.0


def test_clock_summary_without_samples_or_tool(tmp_path, monkeypatch):
    assert _sampler_with(tmp_path, "").summary()["reasons"] == ["no samples"]
    monkeypatch.setenv("PATH", str(tmp_path))          # no nvidia-smi on the path
    s = bench.ClockSampler(0)
    s.path = str(tmp_path / "none.csv")
    with s:
        pass
    assert s.summary() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}


def test_percentile_of_empty_and_small_samples():
    assert bench.percentile([], 50) is None
    assert bench.percentile([3.0], 99) == 3.0
    assert bench.percentile([1.0, 2.0, 3.0, 4.0], 50) == 2.5


def test_host_info_reports_cores_and_model():
    h = bench.host_info()
    assert h["nproc"] >= 1 and 1 <= h["usable"] <= h["nproc"]
    assert h["cpu_model"] is None or isinstance(h["cpu_model"], str)


def test_all_core_oracle_workers_run_the_sample(tmp_path):
    # the all-core CPU baseline: spawned processes load the saved arrays and
    # time the oracle's bounded sample; the pair time combines the pieces
    import multiprocessing as mp

    import numpy as np

    from paper_2608_00760_b300 import inputs
    w = inputs.tissue(17, seed=1)
    for k in ("D", "mu", "q", "w"):
        np.save(str(tmp_path / (k + ".npy")), w[k])
    with mp.get_context("spawn").Pool(2) as pool:
        ts = pool.starmap(bench._oracle_worker, [(str(tmp_path), w["h"])] * 2)
    for t in ts:
        assert all(t[k] > 0 for k in ("fwd", "res", "adj", "grad"))
        assert abs(t["total"] - (t["fwd"] + t["res"] + t["adj"] + t["grad"])) < 1e-6
    t = ts[0]
    assert bench._pair_seconds(t, 3, 2) == (3 * (t["fwd"] + t["res"]) + 2 * (t["adj"] + t["res"]) + t["grad"])
    assert 1 <= bench._all_core_processes((257, 257, 257)) <= bench.host_info()["usable"]
