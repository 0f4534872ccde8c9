"""Host logic of bench.py that decides what a bench line reports (no GPU):
the clock and throttle-reason parsing that rejects a throttled run, the
roofline object's choice of DRAM traffic, and the host core count of the
oracle legs."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


class _FakeProc:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def _sampler(lines):
    s = bench.ClockSampler(0)
    s.proc = _FakeProc()
    s.lines = list(lines)
    return s


def test_clock_sampler_median_max_and_reasons():
    # index, sm, max sm, power, active mask, hw_slowdown, hw_thermal, sw_thermal, sw_power_cap
    lines = ["0, 2070, 2070, 400.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "0, 1980, 2070, 1390.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
             "0, 2070, 2070, 600.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
             "garbage line", ""]
    c = _sampler(lines).stop()
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["samples"] == 3 and c["power_w_max"] == 1390.0
    assert c["reasons"] == ["sw_power_cap"]


def test_clock_sampler_reports_thermal_and_hardware_slowdown():
    lines = ["0, 1500, 2070, 900.0, 0x48, Active, Active, Not Active, Not Active",
             "0, 1400, 2070, 900.0, 0x28, Not Active, Not Active, Active, Not Active"]
    c = _sampler(lines).stop()
    assert c["reasons"] == ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown"]
    assert c["sm_mhz"] == 1450.0


def test_clock_sampler_uses_the_samples_inside_the_region():
    # the first line arrived before the timed region began (start() waits for
    # it); only the later ones count, unless there are none
    lines = ["0, 900, 2070, 150.0, 0x1, Not Active, Not Active, Not Active, Not Active",
             "0, 2070, 2070, 700.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "0, 2050, 2070, 710.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = _sampler(lines)
    s.first = 1
    c = s.stop()
    assert c["samples"] == 2 and c["sm_mhz"] == 2060.0
    s = _sampler(lines[:1])
    s.first = 1
    assert s.stop()["samples"] == 1


def test_clock_sampler_without_nvidia_smi():
    s = bench.ClockSampler(0)
    assert s.stop()["reasons"] == ["nvidia-smi unavailable"]


@pytest.fixture
def fixed_peak(monkeypatch):
    monkeypatch.setattr(bench, "_alu_peak", lambda dev: (40273.92, "test peak"))
    # every capture as if taken of the current sources
    for key, cap in bench.KERNEL_NCU.items():
        monkeypatch.setitem(bench.KERNEL_NCU, key, dict(cap, src=bench.source_hash(cap["sources"])))


def test_roofline_traffic_for_the_captured_workload(fixed_peak):
    cap = bench.KERNEL_NCU["beagle"]
    r = bench._roofline(None, 2000.0, "k", "t", cap["workload"] + ": detail", "beagle", cap["units"])
    assert r["bound"] == "alu" and r["frac"] == pytest.approx(2000.0 / 40273.92)
    assert r["traffic"] == pytest.approx(cap["dram_bytes"])
    assert r["issue_active_ncu"] == cap["issue_active"]


def test_roofline_traffic_scaled_only_where_it_grows_with_the_units(fixed_peak):
    g = bench.KERNEL_NCU["grad"]
    r = bench._roofline(None, 1000.0, "k", "t", "adjoint-16384x1M", "grad", 10 * g["units"])
    assert r["traffic"] == pytest.approx(10 * g["dram_bytes"])  # the tape write-back scales
    assert r["issue_active_ncu"] is None  # not the captured workload
    for key in ("large", "batched"):
        assert not bench.KERNEL_NCU[key]["scale"]
        r = bench._roofline(None, 1000.0, "k", "t", "another-size", key, 1e13)
        assert r["traffic"] is None


def test_roofline_dram_side_of_the_launch(fixed_peak, monkeypatch):
    monkeypatch.setattr(bench, "peaks", lambda: ({"hbm_gbs": 6000.0}, "test"))
    g = bench.KERNEL_NCU["grad"]
    units = 10 * g["units"]
    r = bench._roofline(None, 1000.0, "k", "t", "adjoint-16384x1M", "grad", units)
    seconds = units / 1000.0e9
    assert r["hbm"]["gbs"] == pytest.approx(10 * g["dram_bytes"] / seconds / 1e9)
    assert r["hbm"]["frac"] == pytest.approx(r["hbm"]["gbs"] / 6000.0)
    assert bench._roofline(None, 100.0, "k", "t", "plain-256x1k")["hbm"] is None


def test_roofline_without_a_capture(fixed_peak):
    r = bench._roofline(None, 100.0, "k", "t", "plain-256x1k")
    assert r["traffic"] is None and r["issue_active_ncu"] is None and r["peak"] == 40273.92


def test_stale_capture_is_not_reported(monkeypatch):
    """A capture taken of other kernel sources (or of unknown ones) gives no
    traffic and no issue rate, and says why."""
    monkeypatch.setattr(bench, "_alu_peak", lambda dev: (40273.92, "test peak"))
    cap = bench.KERNEL_NCU["beagle"]
    for src, why in ((None, "no capture"), ("0123456789abcdef", "changed")):
        monkeypatch.setitem(bench.KERNEL_NCU, "beagle", dict(cap, src=src))
        r = bench._roofline(None, 2000.0, "k", "t", cap["workload"], "beagle", cap["units"])
        assert r["traffic"] is None and r["issue_active_ncu"] is None and r["hbm"] is None
        prov = r["ncu_provenance"]
        assert why in prov["stale"] and prov["capture"] == cap["capture"]
        assert prov["src_now"] == bench.source_hash("eval")


def test_source_hash_follows_the_kernel_files():
    assert bench.source_hash("eval") != bench.source_hash("grad")
    assert len(bench.source_hash("eval")) == 16


def test_host_cores_is_the_affinity():
    n = bench.host_cores()
    assert n >= 1
    if hasattr(os, "sched_getaffinity"):
        assert n == len(os.sched_getaffinity(0))
