"""Host-side logic of bench.py (no GPU): the per-stage byte accounting and the
rule that reports ncu DRAM traffic only for the kernel sources it was taken on."""
import os

import pytest

import bench


def test_stage_bytes_add_up_to_the_call():
    """At Nq = 20 on 180 points along x the stages move 766 B per grid point
    (117 + 160.9 + 161.8 + 298.1 + 16.2 + 12.0), against the 396 B/pt floor."""
    sb = bench.stage_bytes_per_point(20, 180)
    assert set(sb) == {"pointwise", "theta_plane", "pencil_contract", "energy_final", "assemble", "pencil_div",
                       "div_final"}
    h = 91 / 180
    assert sb["pointwise"] == pytest.approx(117)
    assert sb["pencil_contract"] == pytest.approx(2 * 20 * 8 * h)
    assert sum(sb.values()) == pytest.approx(766.0, abs=0.1)
    assert bench.b_alg(20) == 396 < sum(sb.values())


def test_traffic_reported_only_for_matching_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_0812_0244_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cu").write_text("kernel one")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.source_sha1()
    (tmp_path / "profiles" / "dram_traffic_dwnt_180x180x72_nq20.txt").write_text(
        "# comment\nsource_sha1 %s\npencil_contract 123456\n" % sha)
    assert bench.captured_traffic("pencil_contract") == 123456
    assert bench.captured_traffic("assemble") is None  # not captured
    (csrc / "a.cu").write_text("kernel two")               # sources changed since the capture
    assert bench.source_sha1() != sha
    assert bench.captured_traffic("pencil_contract") is None


def test_committed_traffic_file_names_its_sources():
    path = os.path.join(os.path.dirname(bench.__file__), "profiles", "dram_traffic_dwnt_180x180x72_nq20.txt")
    keys = [line.split()[0] for line in open(path) if line.strip() and not line.startswith("#")]
    assert keys[0] == "source_sha1" and "pencil_contract" in keys
