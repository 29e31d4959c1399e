"""Host-side arithmetic of bench.py: the algorithmic bytes behind the
roofline fractions (the per-stage traffic the method must move) and the
DRAM-traffic record keyed to the kernels' sources."""
import json
import os

import pytest

import bench


def test_fine_stage_bytes():
    """Fused stage, mean over the three TVDRK3 stages: read w^(s) and write
    w^(s+1) in every stage, read w^n in stages 2 and 3 (8 + 12 + 12 bytes
    per FP32 unknown over three stages), plus the elliptic-grid psi read and
    the restricted field written (l >= 1) or the fine psi read (l = 0)."""
    N = 2047 * 4095
    Nc = 511 * 1023
    assert bench.alg_bytes_per_launch("fine", 2048, 4096, 2, 4) == pytest.approx(
        4 * N * 32 / 12 + 8 * Nc)
    assert bench.alg_bytes_per_launch("fine", 2048, 4096, 0, 4) == pytest.approx(
        4 * N * 32 / 12 + 4 * N)
    assert bench.alg_bytes_per_launch("fine", 2048, 4096, 2, 4) / 1e6 == pytest.approx(93.6, abs=0.1)


def test_solve_bytes():
    """Six passes over the elliptic grid: read and write in the x pass, the
    y pass and the inverse x pass (24 Nc bytes in FP32, 48 Nc in FP64)."""
    Nc = 511 * 1023
    assert bench.alg_bytes_per_launch("solve", 2048, 4096, 2, 4) == 24 * Nc
    assert bench.alg_bytes_per_launch("solve", 2048, 4096, 2, 8) == 48 * Nc
    assert bench.alg_bytes_per_launch("other", 2048, 4096, 2, 4) is None


def test_traffic_record_is_keyed_to_the_sources(tmp_path, monkeypatch):
    """The committed ncu record fills `traffic` only while its source hash
    matches the kernel's current sources."""
    rec = json.load(open(os.path.join(bench.ROOT, "profiles", "dram_traffic_2048x4096_l2.txt")))
    for cls in ("fine", "solve"):
        ent = rec["kernels"][cls]
        got = bench.ncu_traffic(cls)
        if ent["source_hash"] == bench.kernel_source_hash(cls):
            assert got == ent["bytes_per_launch_full_size"]
        else:
            assert got is None
    # a record taken on other sources is not used
    fake = dict(rec)
    fake["kernels"] = {c: dict(v, source_hash="0" * 16) for c, v in rec["kernels"].items()}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "dram_traffic_2048x4096_l2.txt").write_text(json.dumps(fake))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_source_hash", lambda cls: "1" * 16)
    assert bench.ncu_traffic("fine") is None
