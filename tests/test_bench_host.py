"""Host logic of bench.py that needs no GPU: the recorded DRAM traffic is
reported only while the CUDA sources are those the capture ran."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_traffic_is_reported_only_for_unchanged_sources(monkeypatch):
    key = ("volume", "fp64", 4)
    per_elem, sha, prof = bench.TRAFFIC[key]
    monkeypatch.setattr(bench, "_sources_sha", lambda: sha)
    t, src = bench.traffic_of(*key, 1000)
    assert t == per_elem * 1000 and src == prof
    monkeypatch.setattr(bench, "_sources_sha", lambda: "0" * 64)
    t, why = bench.traffic_of(*key, 1000)
    assert t is None and "changed" in why
    t, why = bench.traffic_of("grad", "fp64", 4, 1000)
    assert t is None


def test_sources_hash_covers_the_cuda_sources(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2408_16509_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text("x")
    (csrc / "b.cpp").write_text("y")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench._sources_sha()
    (csrc / "b.cpp").write_text("z")           # host source: not hashed
    assert bench._sources_sha() == h0
    (csrc / "a.cuh").write_text("x2")
    assert bench._sources_sha() != h0
