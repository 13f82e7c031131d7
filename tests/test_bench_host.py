"""bench.py's host-side logic, on the CPU: the algorithmic bytes its roofline
divides by (worked by hand for the power-law LP), the rule that DRAM traffic
from profiles/traffic.json is reported only for the kernel sources it was
taken on, the clock-sample summary that decides whether a run is kept, and
the reference arm's JSON line (the oracle on the small planted LP)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_by_hand():
    # m = 200,000, n = 1,000,000, nnz = 5,000,000, float32 (s = 4):
    # primal: 5e6 (4 + 4) + 4 (1e6 + 1) + 4 (2e5 + 5e6) = 40e6 + 4,000,004 + 20.8e6
    # dual:   5e6 (4 + 4) + 4 (2e5 + 1) + 4 (1e6 + 9 * 2e5) = 40e6 + 800,004 + 11.2e6
    ab = bench.algorithmic_bytes(200_000, 1_000_000, 5_000_000, 4)
    assert ab == {"primal": 64_800_004, "dual": 52_000_004}
    # float64 doubles the value and vector bytes, not the indices
    ab8 = bench.algorithmic_bytes(200_000, 1_000_000, 5_000_000, 8)
    assert ab8["primal"] == 5_000_000 * 12 + 4_000_004 + 8 * 5_200_000


def test_traffic_is_reported_only_for_its_kernel_sources(monkeypatch):
    d = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    key = "powerlaw/fp32/panel_primal/Epanels"
    e = d[key]
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: e["source_sha"])
    assert bench.ncu_traffic("panel_primal", "fp32", "powerlaw", "panels") == e["bytes_per_launch"]
    monkeypatch.setattr(bench, "kernel_source_sha", lambda: "0" * 16)
    assert bench.ncu_traffic("panel_primal", "fp32", "powerlaw", "panels") is None
    assert bench.ncu_traffic("panel_primal", "fp64", "powerlaw", "panels") is None


def test_kernel_source_sha_ignores_comments(tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_2603_03150_gb300", "csrc")
    files = ["spmv_tile.cuh", "iter_kernels.cu", "common.cuh", "epilogues.cuh", "panel.cu"]
    fake = tmp_path / "paper_2603_03150_gb300" / "csrc"
    fake.mkdir(parents=True)
    for f in files:
        (fake / f).write_text(open(os.path.join(src, f)).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_sha()
    p = fake / "panel.cu"
    p.write_text(p.read_text() + "\n// a comment\n/* another\n comment */\n")
    assert bench.kernel_source_sha() == h0
    p.write_text(p.read_text() + "\nint extra_symbol;\n")
    assert bench.kernel_source_sha() != h0


def _clocks_from(tmp_path, lines):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    open(c.path, "w").write("\n".join(lines) + "\n")
    c.p = object()  # as if nvidia-smi had run
    return c.summary()


def test_clock_summary_median_and_reasons(tmp_path):
    ok = "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active"
    cap = "0, 1980, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active"
    hot = "0, 1500, 2070, 1300.0, 0x40, Not Active, Active, Not Active, Not Active"
    s = _clocks_from(tmp_path, [ok, ok, cap, "garbage", ok])
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0 and s["samples"] == 4
    assert s["reasons"] == ["sw_power_cap"]
    s = _clocks_from(tmp_path, [ok, hot, hot])
    assert s["sm_mhz"] == 1500.0 and s["reasons"] == ["hw_thermal_slowdown"]
    assert _clocks_from(tmp_path, ["garbage"])["reasons"] == ["no samples"]


def test_reference_arm_prints_the_contract_line():
    pytest.importorskip("scipy")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "small", "--steps", "2", "--warmup", "3", "--ref-iters", "8"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "iter/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["metric"] == bench.METRIC
    assert line["steps"] == 2 and line["warmup"] == 3
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "iter/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
