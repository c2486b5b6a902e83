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
import os, sys, time
with open(os.environ["FAKE_SMI_ARGS"], "a") as f:
    f.write(sys.argv[sys.argv.index("-i") + 1] + "\\n")
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


def run_region(monkeypatch, path, warm=0.3, region=0.15, gpu="GPU-0b1c2d3e-aaaa-bbbb-cccc-000000000000"):
    import bench
    monkeypatch.setenv("PATH", path + os.pathsep + os.environ.get("PATH", ""))
    monkeypatch.setenv("FAKE_SMI_ARGS", os.path.join(os.path.dirname(path), "args.txt"))
    c = bench.ClockSampler(gpu)
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


def test_gpu_selected_by_uuid(tmp_path, monkeypatch):
    # nvidia-smi ignores CUDA_VISIBLE_DEVICES: the sampler must name the GPU it
    # was given (a UUID) in its -i argument, not a CUDA ordinal
    path = fake_smi(tmp_path, LOOP.format(refuse_50=False, cap_until=0))
    run_region(monkeypatch, path, gpu="GPU-12345678-9abc-def0-1234-56789abcdef0")
    args = open(tmp_path / "args.txt").read().split()
    assert args and set(args) == {"GPU-12345678-9abc-def0-1234-56789abcdef0"}


def test_selector_maps_visible_devices(monkeypatch):
    # without a UUID the ordinal maps through CUDA_VISIBLE_DEVICES to the physical index
    import bench
    import torch
    monkeypatch.setattr(torch.cuda, "get_device_properties", lambda d: (_ for _ in ()).throw(RuntimeError()))
    monkeypatch.setenv("CUDA_VISIBLE_DEVICES", "5,2")
    assert bench.gpu_selector("cuda:1", 1) == "2"
    assert bench.gpu_selector("cuda:0", 0) == "5"
    monkeypatch.delenv("CUDA_VISIBLE_DEVICES")
    assert bench.gpu_selector("cuda:0", 0) == "0"
