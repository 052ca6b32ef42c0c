"""Host-side helpers of bench.py (no GPU): the recorded-traffic lookup keyed by
the kernel source's hash, and the clock sampler's parsing of nvidia-smi
output, exercised with a stand-in nvidia-smi on PATH."""
import os
import stat
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_recorded_traffic_follows_the_source_hash(tmp_path):
    sha = bench.src_sha("iter.cu")
    f = tmp_path / "traffic.txt"
    f.write_text("# comment line\n"
                 f"spmm_hop:dcsbm src_sha={sha} dram_bytes=12345\n"
                 "spmm_hop:other src_sha=0000000000000000 dram_bytes=1\n")
    assert bench.recorded_traffic(str(f), "spmm_hop:dcsbm", "iter.cu") == 12345
    assert bench.recorded_traffic(str(f), "spmm_hop:other", "iter.cu") is None      # stale hash
    assert bench.recorded_traffic(str(f), "spmm_hop:missing", "iter.cu") is None
    assert bench.recorded_traffic(str(tmp_path / "absent.txt"), "spmm_hop:dcsbm", "iter.cu") is None


def _fake_smi(tmp_path, lines):
    script = tmp_path / "nvidia-smi"
    body = "\n".join(f"echo '{ln}'; sleep 0.02" for ln in lines)
    script.write_text("#!/bin/bash\n" + body + "\nexec sleep 30\n")
    script.chmod(script.stat().st_mode | stat.S_IXUSR)
    return str(tmp_path)


@pytest.mark.parametrize("power_cap", [False, True])
def test_clock_sampler_keeps_the_timed_window(tmp_path, monkeypatch, power_cap):
    import datetime
    import time
    cap = "Active" if power_cap else "Not Active"
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)
    stamps = [base + datetime.timedelta(seconds=s_) for s_ in range(6)]
    mhz = [1400, 2070, 2055, 2070, 1980, 1500]     # the first and last samples lie outside the window
    lines = [f"{t.strftime('%Y/%m/%d %H:%M:%S')}.000, 0, {m}, 2070, 1200.5, 0x0, Not Active, Not Active, "
             f"Not Active, {cap}" for t, m in zip(stamps, mhz)]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    c = bench.Clocks(0)
    time.sleep(0.4)
    out = c.stop(stamps[1].timestamp(), stamps[4].timestamp())
    assert out["samples"] == 4
    assert out["sm_mhz"] == 2062.5 and out["sm_max_mhz"] == 2070.0
    assert out["power_w_max"] == 1200.5
    assert out["reasons"] == (["sw_power_cap"] if power_cap else [])
    c = bench.Clocks(0)
    time.sleep(0.4)
    assert c.stop()["samples"] == 6                 # no window: every sample
