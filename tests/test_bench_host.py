"""bench.py host logic without a GPU: the workload table and the source-hash gate on ncu traffic."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import bench  # noqa: E402


def test_workloads_are_complete():
    kinds = {"cg", "mixed32", "mrhs", "batched", "wilson", "full", "force"}
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


def test_default_workload_is_the_32_4_mixed_solve():
    wl = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]
    assert wl["kind_solve"] == "mixed32" and wl["dims"] == (32, 32, 32, 32)
    assert wl["inner"] == "half12" and wl["mass"] == 0.01 and wl["tol"] == 1e-10


def test_default_line_batched_legs_run_at_the_headline_precision():
    head = bench.WORKLOADS[bench.DEFAULT_WORKLOAD]["inner"]
    kinds = set()
    for key in bench.BATCHED_LEGS:
        wl = bench.WORKLOADS[key]
        kinds.add(wl["kind_solve"])
        assert wl["inner"] == head and wl["tol"] == 1e-10
    assert kinds == {"mrhs", "batched"}
    assert bench.WORKLOADS["mrhs24_half12"]["nrhs"] == 16 and bench.WORKLOADS["batch64_half12"]["n"] == 64


def test_k1_k2_bytes_match_the_per_site_table():
    # FP64 K1 = 1152 + 2*48, K2 = 1152 + 48 + 2*48 + 48 + 48 + 48; FP32 recon-12 and FP16 recon-12
    assert bench._k1_k2_bytes("double") == (1248, 1440)
    assert bench._k1_k2_bytes("single12") == (432, 528)
    assert bench._k1_k2_bytes("half12") == (224, 304)
    # the FP32 K1 with p = r + beta p folded in: links + r + p_old read + p + ap written
    assert bench._k1_k2_bytes("single12", folded=True) == (480, 528)


def test_oracle_pool_applies_a_over_every_even_site_on_several_processes():
    """The all-core oracle baseline: one spawned process per core, each applying the oracle's A to
    a slice of the even sites; together they cover the lattice once per pass."""
    from oracle import staggered as S
    from paper_1311_2719_gb300 import inputs as I
    dims = (4, 4, 4, 4)
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    pool = bench.OraclePool(U, b, dims, 0.1, cores=2)
    try:
        flops, dt = pool.run_pass()
    finally:
        pool.close()
    assert pool.cores == 2 and pool.n_even == S.volume(dims) // 2
    assert sorted(np.concatenate(pool.slices).tolist()) == np.nonzero(S.parity(dims) == 0)[0].tolist()
    assert flops == 2 * bench.FLOP_PER_SITE * pool.n_even and dt > 0
    assert bench._oracle_worker_apply  # importable by the spawned workers


def test_sampled_oracle_residual_of_an_exact_solution_is_its_scale():
    """x = (1 - eps) A^-1 b leaves b - A x = eps b at every site: the sampled residual is eps."""
    from oracle import staggered as S
    from paper_1311_2719_gb300 import inputs as I
    dims, m, eps = (4, 4, 4, 4), 0.5, 1e-3
    U = I.make_links(dims, kind="haar", seed=1)
    b = I.make_source(dims, seed=2)
    ref = S.cg_solve(U, b, dims, m, tol=1e-14, max_iter=2000)
    got = bench.sampled_oracle_residual(U, (1 - eps) * ref["x"], b, dims, m, n_sites=40)
    assert abs(got - eps) <= 1e-10
