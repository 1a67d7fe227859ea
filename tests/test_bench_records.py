"""The committed ncu record that bench.py reads: it is keyed by a hash of the step-kernel sources,
so a record taken on another source is never reported, and the roofline objects built from it are
the arithmetic they claim (no GPU needed)."""
import json
import os
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_record_is_consistent_and_reported_only_for_its_source():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as fh:
        rec = json.load(fh)
    if rec["source_hash"] != bench.kernel_source_hash():  # taken on another source: never reported
        assert bench.ncu_traffic("fp32", 256) is None
        return
    for prec, ent in rec["entries"].items():
        if "bytes_per_cell" not in ent:  # an instruction-count entry only
            assert bench.ncu_traffic(prec, 256) is None
            continue
        b = bench.BYTES[prec]
        # the DRAM traffic of a launch is the algorithmic 27 loads and (up to what stays in L2) 27
        # stores per cell
        assert ent["read_bytes_per_cell"] == pytest.approx(27 * b, rel=2e-3)
        assert 0.9 * 27 * b <= ent["write_bytes_per_cell"] <= 27 * b * 1.002
        assert ent["bytes_per_cell"] == pytest.approx(ent["read_bytes_per_cell"] + ent["write_bytes_per_cell"],
                                                      abs=0.02)
    assert bench.ncu_traffic("fp32", 256) == pytest.approx(rec["entries"]["fp32"]["bytes_per_cell"] * 256 ** 3)


def test_record_is_ignored_after_a_kernel_source_change(monkeypatch, tmp_path):
    src = os.path.join(ROOT, "paper_2410_09739_gb300", "csrc")
    copy = tmp_path / "paper_2410_09739_gb300" / "csrc"
    shutil.copytree(src, copy)
    with open(copy / "collide.cuh", "a") as fh:
        fh.write("\n// edited\n")
    (tmp_path / "profiles").mkdir()
    shutil.copy(os.path.join(ROOT, "profiles", "ncu_traffic.json"), tmp_path / "profiles")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.ncu_traffic("fp32", 256) is None
    assert bench.alu_roofline("bf16", 49000.0) is None


def test_alu_roofline_arithmetic():
    alu = bench.alu_roofline("bf16", 50000.0)
    if alu is None:  # the record was taken on another kernel source
        assert bench.ncu_entry("bf16") is None
        return
    assert alu["bound"] == "alu"
    assert alu["peak"] == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    assert alu["achieved"] == pytest.approx(50000.0e6 * alu["lane_ops_per_cell"] / 1e12)
    assert alu["frac"] == pytest.approx(alu["achieved"] / alu["peak"])
    assert bench.alu_roofline("fp64", 1000.0) is None  # no record for that storage type
