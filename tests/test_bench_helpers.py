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
def test_clock_sampler_parses_every_sample(tmp_path, monkeypatch, power_cap):
    cap = "Active" if power_cap else "Not Active"
    lines = [f"0, {mhz}, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, {cap}"
             for mhz in (2070, 2055, 2070, 1980, 2070)]
    monkeypatch.setenv("PATH", _fake_smi(tmp_path, lines) + os.pathsep + os.environ["PATH"])
    c = bench.Clocks(0)
    assert c.first.startswith("0, 2070")        # the first sample is read before timing starts
    import time
    time.sleep(0.3)
    out = c.stop()
    assert out["samples"] == 5                  # the first sample is counted with the rest
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["power_w_max"] == 1200.5
    assert out["reasons"] == (["sw_power_cap"] if power_cap else [])
