"""Host logic of the bench line that needs no GPU: the DRAM-traffic figure
is taken from a committed ncu summary only while the count kernels' sources
still hash to the value recorded in it, and only for its own workload."""
from __future__ import annotations

import bench


def write_profile(tmp_path, sha, workload, read_gb, write_gb):
    p = tmp_path / ("count_dram_traffic_%s.md" % workload)
    p.write_text("# x\n\nworkload: %s\nsource-sha256: %s\n\n| kernel | read GB | write GB | ms |\n|---|---|---|---|\n"
                 "| count_bitmap_s | %s | %s | 1.0 |\n| count_warp | 1.5 | 0.5 | 1.0 |\n"
                 % (workload, sha, read_gb, write_gb))
    return p


def test_traffic_read_only_for_current_sources(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "traffic_profile", lambda wl: str(tmp_path / ("count_dram_traffic_%s.md" % wl)))
    sha = bench.count_sources_sha()
    write_profile(tmp_path, sha, "rmat-s24-ef16", "120.5", "8.25")
    assert bench.dram_traffic("count_bitmap_s", "rmat-s24-ef16") == (120.5 + 8.25) * 1e9
    assert bench.dram_traffic("count_warp", "rmat-s24-ef16") == 2.0e9
    assert bench.dram_traffic("count_thread", "rmat-s24-ef16") is None       # no row
    assert bench.dram_traffic("count_bitmap_s", "rmat-s22-ef16") is None     # no file
    write_profile(tmp_path, "0" * 64, "rmat-s24-ef16", "120.5", "8.25")      # other sources
    assert bench.dram_traffic("count_bitmap_s", "rmat-s24-ef16") is None


def test_traffic_profile_names_its_workload(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "traffic_profile", lambda wl: str(tmp_path / "count_dram_traffic_rmat-s24-ef16.md"))
    write_profile(tmp_path, bench.count_sources_sha(), "rmat-s22-ef16", "9.7", "0.4")
    assert bench.dram_traffic("count_bitmap_s", "rmat-s24-ef16") is None
