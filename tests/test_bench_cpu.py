"""CPU checks of the benchmark's roofline bookkeeping: the algorithmic work per element, the executed-work
figure, and the captured ncu counters, which the bench line reports only while the kernel source they were
taken from is unchanged."""
import os

import pytest

import bench
import workloads


def test_algorithmic_ops_per_element():
    # d projection FMAs, 3 ops per histogram pass of the two selections, 2 more for the D_AP count
    assert bench.alu_ops_per_element(workloads.PROJECTION, 10) == 16
    assert bench.alu_ops_per_element(workloads.ASYM_PROJECTION, 10) == 18
    assert bench.alu_ops_per_element(workloads.PROJECTION, 1) == 7


def test_captured_counters_follow_the_kernel_source(monkeypatch):
    for key, entry in bench.CAPTURED.items():
        for f in entry["src"]:
            assert os.path.exists(os.path.join(bench.ROOT, f)), f
        live = bench.src_sha16(entry["src"])
        # same source: the stored value; any other source: nothing
        monkeypatch.setitem(bench.CAPTURED, key, dict(entry, src_sha16=live))
        assert bench.captured(key, "traffic") == entry["traffic"]
        monkeypatch.setitem(bench.CAPTURED, key, dict(entry, src_sha16="0" * 16))
        assert bench.captured(key, "traffic") is None
        monkeypatch.setitem(bench.CAPTURED, key, dict(entry, src_sha16=None))
        assert bench.captured(key, "traffic") is None
        monkeypatch.setitem(bench.CAPTURED, key, entry)


def test_source_hash_covers_every_byte(tmp_path, monkeypatch):
    a = tmp_path / "a.cu"
    a.write_text("__global__ void k() {}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h1 = bench.src_sha16(["a.cu"])
    a.write_text("__global__ void k() {}\n// note\n")
    assert bench.src_sha16(["a.cu"]) != h1
    assert len(h1) == 16


def test_executed_work_against_the_issue_peak(monkeypatch):
    entry = dict(bench.CAPTURED["k_pdap2_c2"])
    entry["src_sha16"] = bench.src_sha16(entry["src"])
    entry["warp_instr_per_element"] = 2.0
    monkeypatch.setitem(bench.CAPTURED, "k_pdap2_c2", entry)
    # 5e8 elements x 2 warp instructions in 1 ms: 1e12 warp instructions per second
    ex = bench.executed_work(True, 5e8, 1.0)
    assert ex["achieved_warp_instr_per_s"] == pytest.approx(1e12)
    peak = 152 * 4 * 2070e6
    assert ex["peak_warp_instr_per_s"] == pytest.approx(peak)
    assert ex["frac"] == pytest.approx(1e12 / peak)
    # a launch shape other than the captured one has no executed-work figure
    assert bench.executed_work(False, 5e8, 1.0) is None
