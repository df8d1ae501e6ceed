"""bench.py's host-side helpers on the CPU: the algorithmic byte counts
(per-unit figures times units) and the rule that a committed ncu capture is
used only while the kernel source it was taken on is unchanged."""
import hashlib
import json
import math

import bench


def test_diffusion_bytes_are_the_per_unit_figures_times_the_units():
    # 16 V + 16 E per sweep: per vertex a row pointer, the diagonal, u read and
    # written (4 each); per directed edge (2E) a column index and a weight (8)
    assert bench.gs_bytes(1_050_625, 3_147_776, 2000) == 2000 * (16 * 1_050_625 + 8 * 2 * 3_147_776)
    assert bench.gs_bytes(1_050_625, 3_147_776, 2000) == 134_348_832_000
    # the 168M-vertex mesh: 4000 x (16 x 167,772,162 + 16 x 503,316,480) = 42.95 TB per launch
    assert bench.gs_bytes(167_772_162, 503_316_480, 4000) == 42_949_673_088_000
    # the library's 8-byte state adds 8 bytes per vertex-sweep
    assert bench.gs_state_bytes(1_050_625, 2000) == 2000 * 8 * 1_050_625


def test_traffic_scales_with_vertex_sweeps():
    cap = {"dram_bytes_per_launch": 1.0e9, "vertex_sweeps": 2_621_442 * 100}
    t = bench.scaled_traffic(cap, 167_772_162, 4000)
    assert math.isclose(t, 1.0e9 * 167_772_162 * 4000 / (2_621_442 * 100))
    assert bench.scaled_traffic(None, 10, 10) is None


def test_stage_bytes():
    nv, ne, nf = 1000, 2970, 1971
    face = bench.stage_bytes(nv, ne, nf, 10, 10, "face", 100)
    edge = bench.stage_bytes(nv, ne, nf, 10, 10, "edge", 100)
    assert face["diffusion"] == edge["diffusion"] == bench.gs_bytes(nv, ne, 10)
    assert face["normalize"] == 66 * nf
    assert face["admm"] == 10 * 154 * nf - 48 * nf
    assert bench.stage_bytes(nv, ne, nf, 10, 1, "face", 100)["admm"] == 106 * nf
    assert edge["admm"] == 78 * nf + 32 * ne + 10 * (69 * nf + 40 * ne)
    rounds = math.ceil(math.log2(100))
    assert face["integrate"] == 88 * nv + 24 * nv * rounds
    assert edge["integrate"] == 40 * nv + 24 * nv * rounds
    assert face["bfs_layout"] == 88 * nv + 52 * 2 * ne


def test_capture_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    src = tmp_path / "paper_1812_06060_gb300" / "csrc"
    src.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    (src / "gs.cu").write_bytes(b"// kernel v1\n")
    rec = {"dram_bytes_per_full_launch": 123.0, "lts_bytes": 456.0,
           "gs_cu_sha256": hashlib.sha256(b"// kernel v1\n").hexdigest()}
    (tmp_path / "profiles" / "k_gs_grid1025.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.capture("k_gs_grid1025")["dram_bytes_per_full_launch"] == 123.0
    assert bench.capture("k_gs_grid1025")["lts_bytes"] == 456.0
    assert bench.capture("k_gs_sinusoid_ico9") is None
    (src / "gs.cu").write_bytes(b"// kernel v2\n")
    assert bench.capture("k_gs_grid1025") is None
