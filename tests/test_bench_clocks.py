"""The benchmark's clock sampler, against a stand-in for nvidia-smi on PATH (no
GPU): only the samples taken inside the timed region count, throttle reasons are
read from the flag columns, the 200 ms period is the fallback when a 50 ms loop
gives nothing, and a missing tool yields None instead of an exception."""
import os
import stat
import sys
import time

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def fake_smi(tmp_path, body):
    d = tmp_path / "bin"
    d.mkdir()
    f = d / "nvidia-smi"
    f.write_text("#!" + sys.executable + "\n" + body)
    f.chmod(f.stat().st_mode | stat.S_IXUSR)
    return str(d)


LOOP = """
import sys, time
period = 0.05 if "50" in sys.argv else 0.2
if "50" in sys.argv and {refuse_50}:
    sys.exit(2)
i = 0
t0 = time.time()
while True:
    cap = "Active" if time.time() - t0 < {cap_until} else "Not Active"
    print(f"0, {{2070 - i % 2}}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {{cap}}", flush=True)
    i += 1
    time.sleep(period)
"""


def run_region(monkeypatch, path, warm=0.3, region=0.15):
    import bench
    monkeypatch.setenv("PATH", path + os.pathsep + os.environ.get("PATH", ""))
    c = bench.ClockSampler(0)
    c.start()
    time.sleep(warm)  # outside the timed region
    c.mark()
    time.sleep(region)
    return c.stop()


def test_samples_inside_the_region_only(tmp_path, monkeypatch):
    # power capping reported only during the first 0.2 s, before the region
    path = fake_smi(tmp_path, LOOP.format(refuse_50=False, cap_until=0.2))
    r = run_region(monkeypatch, path)
    assert r is not None and r["period_ms"] == 50
    assert 1 <= r["samples"] <= 8
    assert r["reasons"] == [] and r["sm_max_mhz"] == 2070.0 and 2069.0 <= r["sm_mhz"] <= 2070.0


def test_reasons_seen_inside_the_region(tmp_path, monkeypatch):
    path = fake_smi(tmp_path, LOOP.format(refuse_50=False, cap_until=60))
    r = run_region(monkeypatch, path)
    assert r["reasons"] == ["sw_power_cap"]


def test_fallback_period(tmp_path, monkeypatch):
    path = fake_smi(tmp_path, LOOP.format(refuse_50=True, cap_until=0))
    r = run_region(monkeypatch, path, warm=0.1, region=0.25)
    assert r is not None and r["period_ms"] == 200 and r["samples"] >= 1


def test_missing_tool_gives_none(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))
    c = bench.ClockSampler(0)
    c.start()
    c.mark()
    assert c.stop() is None
