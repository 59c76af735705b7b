"""Host-side arithmetic of bench.py, on fake inputs: the nvidia-smi clock
record (median SM clock, throttle reasons) and the contraction GB/s of the
roofline object (algorithmic bytes over CUDA-event time).  CPU only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _line(sm, mx=2070, act="0x0000000000000000", hw="Not Active", hwt="Not Active",
          swt="Not Active", cap="Not Active"):
    return f"0, {sm}, {mx}, 900.5, {act}, {hw}, {hwt}, {swt}, {cap}"


def test_clock_lines_median_and_reasons():
    lines = [_line(1965), _line(2032, cap="Active"), _line(1980), "garbage", "",
             _line("[N/A]"), _line(1990, mx="[N/A]"), _line(1700, hwt="Active")]
    c = bench.parse_clock_lines(lines)
    assert c["samples"] == 4
    assert c["sm_mhz"] == pytest.approx((1965 + 1980) / 2)
    assert c["sm_max_mhz"] == 2070
    assert c["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_clock_lines_empty():
    assert bench.parse_clock_lines([]) is None
    assert bench.parse_clock_lines(["a, b"]) is None


def test_contraction_gbs_is_algorithmic_bytes_over_time():
    prof = {
        "contract_rows": {"ms": 2.0, "units": 10**9, "launches": 4},
        "emit": {"ms": 1.0, "units": 10**8, "launches": 1},
        "sort_pass": {"ms": 0.0, "units": 5, "launches": 0},  # not run: skipped
        "pr_marks": {"ms": 9.0, "units": 10**9, "launches": 1},  # not contraction
    }
    out = bench.contraction_gbs(prof, 8000.0, "measured")
    b_rows = 10**9 * bench.ALG_BYTES["contract_rows"]
    b_emit = 10**8 * bench.ALG_BYTES["emit"]
    assert out["contract_rows"]["gbs"] == pytest.approx(b_rows / 2e-3 / 1e9)
    assert out["emit"]["gbs"] == pytest.approx(b_emit / 1e-3 / 1e9)
    assert "sort_pass" not in out and "pr_marks" not in out
    tot = (b_rows + b_emit) / 3e-3 / 1e9
    assert out["total"]["gbs"] == pytest.approx(tot)
    assert out["total"]["frac"] == pytest.approx(tot / 8000.0)
    assert out["total"]["peak_kind"] == "measured"
    assert bench.contraction_gbs({}, 8000.0, "measured") == {}


def test_peaks_file_is_read():
    peak, kind = bench.load_peaks()
    assert peak > 0 and kind in ("measured", "fallback")


def test_reference_arm_line_on_cpu():
    """The reference arm (the CPU oracle's NOI) prints the contract's JSON
    line; run here on the small G(2000, 16000) workload."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "er2000", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3
    assert d["config"]["lambda"] == 23
    assert d["value"] > 0 and d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def test_kernel_table_shares_and_algorithmic_rates():
    prof = {"pr_marks": {"ms": 6.0, "units": 3 * 10**9, "launches": 3},
            "union_find": {"ms": 2.0, "units": 0, "launches": 12}}
    t = bench.kernel_table(prof, 2, 8000.0)
    assert list(t) == ["pr_marks", "union_find"]  # by time
    assert t["pr_marks"]["ms_per_step"] == 3.0 and t["pr_marks"]["share"] == 0.75
    gbs = 3 * 10**9 * bench.ALG_BYTES["pr_marks"] / 6e-3 / 1e9
    assert t["pr_marks"]["alg_gbs"] == pytest.approx(gbs)
    assert t["pr_marks"]["frac"] == pytest.approx(gbs / 8000.0)
    assert "alg_gbs" not in t["union_find"]  # no algorithmic byte count
    assert bench.kernel_table({}, 1, 8000.0) == {}


def test_roofline_of_dominant_kernel_traffic_and_note():
    # pr_marks has the longest time among the categories with a byte count
    # (union_find has none and is ignored even though it is listed)
    prof = {"pr_marks": {"ms": 3.0, "units": 3 * 29031216, "launches": 3},
            "contract_rows": {"ms": 2.0, "units": 4 * 10**7, "launches": 4},
            "union_find": {"ms": 9.0, "units": 0, "launches": 12}}
    r = bench.roofline_of(prof, 6776.3, "measured")
    assert r["kernel"] == "pr_marks" and r["bound"] == "hbm" and r["unit"] == "GB/s"
    alg = 29031216 * bench.ALG_BYTES["pr_marks"]  # per launch
    assert r["alg_bytes_per_launch"] == pytest.approx(alg)
    assert r["avg_launch_ms"] == pytest.approx(1.0)
    assert r["achieved"] == pytest.approx(alg / 1e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6776.3)
    # traffic: the captured DRAM bytes per entry, scaled to a launch's entries
    assert r["traffic"] == pytest.approx(bench.TRAFFIC_PER_UNIT["pr_marks"] * 29031216)
    assert "note" not in r
    # a latency-bound category carries its note, and no traffic without a capture
    prof = {"capforest_seq": {"ms": 5000.0, "units": 2 * 169364222, "launches": 2},
            "pr_marks": {"ms": 8.0, "units": 10**8, "launches": 10}}
    r = bench.roofline_of(prof, 6776.3, "measured")
    assert r["kernel"] == "capforest_seq" and r["traffic"] is None
    assert "latency-bound" in r["note"]
    assert bench.roofline_of({"union_find": {"ms": 1.0, "units": 0, "launches": 1}},
                             6776.3, "measured") is None
