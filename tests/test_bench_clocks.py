"""The benchmark's clock record (sampled with nvidia-smi during the timed
region) parsed from a stand-in nvidia-smi that prints known rows: median SM
clock, maximum clock, the throttle reasons that were active, unparsable rows
skipped, and an empty record when nvidia-smi is missing."""
import importlib.util
import os
import stat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


ROWS = """2070, 2070, 900.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
2055, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active
[N/A], 2070, 0.0, 0x0, Not Active, Not Active, Not Active, Not Active
2065, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active
"""


def test_clock_record_from_nvidia_smi_rows(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/sh\ncat <<'EOF'\n" + ROWS + "EOF\nsleep 30\n")
    fake.chmod(fake.stat().st_mode | stat.S_IEXEC)
    monkeypatch.setenv("PATH", str(tmp_path) + os.pathsep + os.environ.get("PATH", ""))
    bench = load_bench()
    s = bench.ClockSampler("0")
    s.start()
    rec = s.stop()
    assert rec == {"sm_mhz": 2065.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}


def test_clock_record_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    bench = load_bench()
    s = bench.ClockSampler("0")
    s.start()
    assert s.stop() == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
