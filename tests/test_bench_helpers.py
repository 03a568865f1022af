"""Host helpers of bench.py (no GPU): the DRAM-traffic lookup is used only for the sources and the workload
it was captured on, and the clock sampler's parsing of nvidia-smi lines (median SM clock, throttle reasons)."""
import json

import bench


def write_traffic(tmp_path, source_hash, workload):
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps({
        "source_hash": source_hash, "workload": workload,
        "stage_dram_bytes_per_iteration": {"factorisation": 1234, "s_build": 99}}))


def test_traffic_only_for_its_sources_and_workload(tmp_path, monkeypatch):
    write_traffic(tmp_path, "abc", "c1_internet, bench.py --steps 2")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "source_hash", lambda: "abc")
    assert bench.stage_traffic("factorisation", "c1_internet") == 1234
    assert bench.stage_traffic("s_build", "c1_internet") == 99
    assert bench.stage_traffic("factorisation", "c4_large") is None      # another workload
    assert bench.stage_traffic("factorisation", "c1") is None            # a prefix of the name is not the name
    monkeypatch.setattr(bench, "source_hash", lambda: "other")
    assert bench.stage_traffic("factorisation", "c1_internet") is None   # the kernels changed since


def test_traffic_absent(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.stage_traffic("factorisation", "c1_internet") is None


class _DoneProcess:
    def terminate(self):
        pass

    def wait(self, timeout=None):
        return 0


def test_clock_sampler_parses_median_and_reasons(tmp_path):
    p = tmp_path / "clocks.csv"
    p.write_text("0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active\n"
                 "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active\n"
                 "garbage line\n")
    cs = bench.ClockSampler(0)
    cs.proc, cs.path = _DoneProcess(), str(p)
    out = cs.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    assert not p.exists()


def test_clock_sampler_without_nvidia_smi():
    assert bench.ClockSampler(0).stop() is None
