"""bench.py host logic without a GPU: the workload table and the source-hash gate on ncu traffic."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_workloads_are_complete():
    kinds = {"cg", "mrhs", "batched", "wilson", "full", "force"}
    for name, wl in bench.WORKLOADS.items():
        assert wl["desc"], name
        assert wl.get("kind_solve", "cg") in kinds, name
        if wl.get("kind_solve") == "wilson":
            assert wl.get("outer", "double") in ("double", "df64"), name
            assert 0.0 < wl.get("reliable_delta", 0.1) < 1.0, name
            if "traffic_key" in wl:  # the same K1/K2 kernels as a captured workload
                key = bench.WORKLOADS[wl["traffic_key"]]
                assert (key["dims"], key["nrhs"], key["inner"]) == (wl["dims"], wl["nrhs"], wl["inner"])
    assert bench.DEFAULT_WORKLOAD in bench.WORKLOADS


def _fake_tree(tmp_path, content):
    csrc = tmp_path / "paper_1311_2719_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (csrc / "a.cuh").write_text(content)
    (tmp_path / "profiles").mkdir()
    return csrc


def test_traffic_is_reported_only_for_the_captured_sources(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path, "kernel v1")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.sources_sha(["a.cuh"])
    entries = {"w_cg": {"K1_bytes": 100, "K2_bytes": 300, "sources": ["a.cuh"], "sources_sha256": sha},
               "w_one": {"bytes": 7, "sources": ["a.cuh"], "sources_sha256": sha}}
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(json.dumps({"workloads": entries}))
    assert bench.ncu_traffic("w_cg") == 200          # the mean of K1 and K2
    assert bench.ncu_traffic("w_one") == 7
    assert bench.ncu_traffic("missing") is None
    (csrc / "a.cuh").write_text("kernel v2")         # the kernel changed since the capture
    assert bench.ncu_traffic("w_cg") is None and bench.ncu_traffic("w_one") is None


def test_source_hash_covers_names_and_contents(tmp_path, monkeypatch):
    csrc = _fake_tree(tmp_path, "x")
    (csrc / "b.cuh").write_text("y")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h = bench.sources_sha(["a.cuh", "b.cuh"])
    assert h == bench.sources_sha(["b.cuh", "a.cuh"])  # order-free
    assert h != bench.sources_sha(["a.cuh"])
    (csrc / "b.cuh").write_text("y ")
    assert h != bench.sources_sha(["a.cuh", "b.cuh"])
