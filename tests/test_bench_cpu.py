"""Host-side helpers of bench.py, on the CPU: the clock summary that decides
whether a timed run is valid, the job rate, and the code hash that keys the
committed DRAM-traffic record to the interaction kernel's code."""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def sampler(bench, rows):
    s = bench.ClockSampler(0)
    s.rows = rows
    return s


def row(sm, smax, power, hw="Not Active", hwt="Not Active", swt="Not Active", cap="Not Active"):
    return ["0", str(sm), str(smax), str(power), "0x0", hw, hwt, swt, cap]


def test_clock_summary_median_max_and_reasons(bench):
    s = sampler(bench, [row(2070, 2070, 300.0), row(1900, 2070, 650.5, cap="Active"),
                        row(2070, 2070, 410.0)])
    out = s.summary()
    assert out["sm_mhz"] == 2070.0
    assert out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    assert out["samples"] == 3
    assert out["power_w_max"] == 650.5


def test_clock_summary_flags_thermal_and_missing_samples(bench):
    out = sampler(bench, [row(1500, 2070, 700.0, hwt="Active")]).summary()
    assert out["reasons"] == ["hw_thermal_slowdown"]
    empty = sampler(bench, [["garbage"]]).summary()
    assert empty["samples"] == 0 and empty["reasons"] == ["unsampled"]


def test_job_rate_counts_every_rank(bench):
    # 1E6 targets per rank, 3 steps, 2 ranks in 300 ms -> 2E7 targets/s
    assert bench.job_rate(1_000_000, 3, 2, 300.0) == pytest.approx(2e7)


def test_code_hash_ignores_comments_and_layout(bench, tmp_path):
    a = tmp_path / "a.cu"
    b = tmp_path / "b.cu"
    a.write_text("int f(int x) {\n  return x + 1;  // add one\n}\n")
    b.write_text("// a header comment\nint f(int x) {\n\n      return x + 1;\n}\n")
    assert bench.code_hash(str(a)) == bench.code_hash(str(b))
    b.write_text("int f(int x) {\n  return x + 2;\n}\n")
    assert bench.code_hash(str(a)) != bench.code_hash(str(b))


def test_traffic_record_matches_the_kernel_it_was_taken_on(bench):
    # The committed record carries the hash of the kernel code it was
    # measured on; the bench reports its traffic only while they agree.
    import json
    with open(os.path.join(ROOT, "profiles", "interact_traffic.json")) as f:
        rec = json.load(f)
    assert rec["dram_bytes_per_launch_full_size"] == rec["dram_bytes_read"] + rec["dram_bytes_write"]
    current = bench.interact_code_hash()
    assert bench.interact_traffic() == (rec["dram_bytes_per_launch_full_size"]
                                        if rec["interact_code_sha256"] == current else None)


def test_reference_arm_prints_the_contract_line(bench):
    """`bench.py --impl reference` times the oracle on the host and prints one
    JSON line with the same metric, unit and workload as the GPU arm."""
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                       timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["steps"] == 1 and d["warmup"] == 0
    assert d["config"]["workload"].startswith("uniform_n1e6")
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == bench.host_cores()   # one oracle process per host core
    assert f"{bench.host_cores()} whole target leaves" in d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
