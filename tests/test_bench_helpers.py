"""Host helpers of bench.py that feed the JSON line: the clock sampler's
parsing of nvidia-smi rows (median SM clock, throttle reasons) and the DRAM
traffic read from the committed ncu summary (only for the kernel source and
the lattice the summary was taken on)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


class _Proc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_rows_parsed():
    c = bench.Clocks(0)
    c.f.write("0, 2070, 2070, 950.1, 0x0000000000000000, Not Active, Not Active, Not Active, "
              "Not Active\n")
    c.f.write("0, 1965, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, "
              "Active\n")
    c.f.write("0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n")
    c.f.write("garbage line\n")
    c.p = _Proc()
    out = c.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"],
                   "samples": 3}
    assert not os.path.exists(c.f.name)


def test_clock_sampler_without_nvidia_smi():
    c = bench.Clocks(0)
    assert c.stop() is None  # never started
    os.unlink(c.f.name)


def test_traffic_only_for_the_profiled_source(monkeypatch):
    import re
    txt = open(os.path.join(ROOT, "profiles", "dslash_traffic.md")).read()
    profiled = re.search(r"source_sha256_16:\s*([0-9a-f]+)", txt).group(1)
    value = float(re.search(r"^dslash_f32_12/cg traffic_bytes_per_launch:\s*([0-9.]+)", txt,
                            re.M).group(1))
    t = bench.ncu_traffic("dslash_f32_12/cg")
    if bench.dslash_source_hash() == profiled:
        assert t == pytest.approx(value)
    else:  # kernel source changed since the capture: no traffic figure
        assert t is None
    monkeypatch.setattr(bench, "dslash_source_hash", lambda: profiled)
    assert bench.ncu_traffic("dslash_f32_12/cg") == pytest.approx(value)
    # taken on 24^3 x 48 only: another lattice gets no traffic figure
    assert re.search(r"^lattice:\s*24\^3x48$", txt, re.M)
    monkeypatch.setattr(bench, "LAT", bench.LATTICES["16x32"])
    assert bench.ncu_traffic("dslash_f32_12/cg") is None
    monkeypatch.setattr(bench, "LAT", bench.LATTICES["24x48"])
    monkeypatch.setattr(bench, "dslash_source_hash", lambda: "0000000000000000")
    assert bench.ncu_traffic("dslash_f32_12/cg") is None
