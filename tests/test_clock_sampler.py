"""bench.py's ClockSampler against a stand-in for nvidia-smi (no GPU): the sampler waits
for its first sample before the timed region starts, drops the samples taken before,
parses the clocks and the throttle reasons, and degrades to an empty record when the tool
is missing."""
import os
import stat
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

FAKE = r"""#!{py}
import sys, time
period = 0.05
if "-lms" in sys.argv:
    period = int(sys.argv[sys.argv.index("-lms") + 1]) / 1000.0
time.sleep(0.2)                      # start-up, as the real tool's library load
n = 0
while True:
    # the first sample is the idle clock; later ones are under load, one power-capped
    sm = 600 if n == 0 else 2070
    cap = "Active" if n == 2 else "Not Active"
    print(f"0, {{sm}}, 2070, 400.5, 0x0, Not Active, Not Active, Not Active, {{cap}}", flush=True)
    n += 1
    time.sleep(period)
"""


def fake_tool(tmp_path):
    p = tmp_path / "nvidia-smi"
    p.write_text(FAKE.format(py=sys.executable))
    p.chmod(p.stat().st_mode | stat.S_IEXEC)
    return str(tmp_path)


def test_samples_inside_the_region(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", fake_tool(tmp_path) + os.pathsep + os.environ["PATH"])
    monkeypatch.setattr(bench.ClockSampler, "PERIOD_MS", 50)
    cs = bench.ClockSampler(0)
    t0 = time.perf_counter()
    cs.start()
    assert time.perf_counter() - t0 >= 0.2          # waited for the tool's first sample
    assert cs.skip >= 1
    time.sleep(0.8)                                  # the "timed region": about 16 periods
    out = cs.stop()
    assert out["samples"] >= 4
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0   # idle sample dropped
    assert out["reasons"] == ["sw_power_cap"]
    assert out["power_w_max"] == 400.5


def test_short_region_reports_the_last_sample(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", fake_tool(tmp_path) + os.pathsep + os.environ["PATH"])
    cs = bench.ClockSampler(0)
    cs.start()
    out = cs.stop()                                  # no time between start and stop
    assert out["samples"] >= 1 and out["sm_mhz"] is not None


def test_missing_tool(tmp_path, monkeypatch):
    import bench
    monkeypatch.setenv("PATH", str(tmp_path))        # no nvidia-smi on the path
    cs = bench.ClockSampler(0)
    cs.start()
    out = cs.stop()
    assert out == {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
