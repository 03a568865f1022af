"""Host helpers of bench.py (no GPU): the DRAM-traffic lookup is used only for the sources and the workload
it was captured on, the clock sampler's parsing of nvidia-smi lines (median SM clock, throttle reasons), and
the max over ranks of a multi-process run (two gloo ranks on CPU)."""
import json
import os
import socket

import pytest

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


def _max_worker(rank, world, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        v = bench.max_over_ranks(10.0 + 3.0 * rank)   # the ranks' own step times
        with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
            f.write(repr(v))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_on_two_gloo_ranks(tmp_path):
    pytest.importorskip("torch")
    import torch.multiprocessing as tmp_mp
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as so:
        so.bind(("127.0.0.1", 0))
        port = so.getsockname()[1]
    tmp_mp.start_processes(_max_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    assert [float((tmp_path / f"r{r}.txt").read_text()) for r in range(2)] == [13.0, 13.0]
    assert bench.max_over_ranks(7.5) == 7.5   # no process group: the value itself


def test_stage_roofline_fractions_and_dominant_stage():
    import bench
    info = {"s_lower_elems": 1e6, "nv": 1e5, "factor_flops": 2e9}
    q, n, m = 100_000, 20_000, 100
    alu = {"fp32_tflops": 60.0, "tf32_tflops": 900.0}
    stage_ms = [0.1, 0.2, 0.4, 0.15, 0.1]
    rf = bench.stage_roofline(info, stage_ms, q, n, m, 6000.0, alu, "no_such_workload")
    st = rf["stages"]
    assert list(st) == bench.STAGES
    for nm, t in zip(bench.STAGES, stage_ms):
        e = st[nm]
        assert e["ms"] == t
        assert abs(e["achieved_gbs"] - e["algorithmic_bytes"] / (t / 1e3) / 1e9) < 1e-9 * e["achieved_gbs"]
        assert abs(e["hbm_frac"] - e["achieved_gbs"] / 6000.0) < 1e-12
        assert "traffic_ratio" not in e   # no capture of this workload
    f = st["factorisation"]
    assert abs(f["achieved_tflops"] - 2e9 / 0.4e-3 / 1e12) < 1e-12
    assert abs(f["fp32_frac"] - f["achieved_tflops"] / 60.0) < 1e-12
    assert abs(f["tensor_3xtf32_frac"] - f["achieved_tflops"] / 300.0) < 1e-12
    d = rf["dominant"]
    assert d["stage"] == "factorisation" and d["bound"] == "alu" and d["peak"] == 60.0
    # an HBM-bound dominant stage, and the derived FP32 peak when none was measured
    rf2 = bench.stage_roofline(info, [0.1, 0.9, 0.4, 0.15, 0.1], q, n, m, 6000.0, None, "x")
    assert rf2["dominant"]["stage"] == "s_build" and rf2["dominant"]["bound"] == "hbm"
    assert rf2["stages"]["factorisation"]["fp32_peak_tflops"] == bench.FP32_PEAK_TFLOPS_DERIVED
