"""Host-side helpers of bench.py: the kernel each SpMV family runs (it must
follow the library's dispatch, which the roofline names), the lookup of ncu
traffic figures (only for the same family, tile_dim, kernel, graph and kernel
source), and the workload description."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("family,tile,schedule,kernel", [
    ("spmv_bool", 4, 2, "spmv_k4_kernel"), ("spmv_count", 4, 1, "spmv_k4_kernel"),
    ("spmv_plus", 4, 2, "spmv_k4_kernel"), ("spmv_min_i32", 4, 2, "spmv_k4_kernel"),
    ("spmv_max", 4, 2, "spmv_k4_kernel"), ("spmm_or32", 4, 2, "spmv_k4_kernel"),
    ("spmm_or64", 4, 2, "spmv_chunks_kernel"), ("spmv_plus", 4, 1, "spmv_gather_kernel"),
    ("spmv_plus", 8, 2, "spmv_chunks_kernel"), ("spmv_plus", 16, 1, "spmv_gather_kernel"),
    ("spmv_plus", 32, 1, "spmv_chunks_kernel"), ("spmv_bool", 8, 2, "spmv_chunks_kernel"),
])
def test_kernel_names_follow_the_dispatch(family, tile, schedule, kernel):
    assert bench.spmv_kernel_name(family, tile, schedule) == kernel


def test_traffic_lookup_matches_graph_and_source(tmp_path, monkeypatch):
    src = os.path.join(ROOT, "paper_2201_08560_gb300", "csrc", "spmv.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    rec = {"a": {"family": "spmv_plus", "tile_dim": 4, "graph": "rmat20", "kernel": "spmv_k4_kernel<SemPlus<4>>",
                 "dram_bytes_per_launch": 123, "kernel_source_sha256": sha},
           "b": {"family": "spmv_plus", "tile_dim": 4, "graph": "rmat20_perm2", "kernel": "spmv_k4_kernel<SemPlus<4>>",
                 "dram_bytes_per_launch": 456, "kernel_source_sha256": "0" * 64}}
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(rec))
    (tmp_path / "paper_2201_08560_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_2201_08560_gb300" / "csrc" / "spmv.cu").write_bytes(open(src, "rb").read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_for("spmv_plus", 4, "spmv_k4_kernel", "rmat20")[0] == 123.0
    assert bench.traffic_for("spmv_plus", 4, "spmv_k4_kernel", "rmat20_perm2")[0] is None  # stale source
    assert bench.traffic_for("spmv_plus", 8, "spmv_k4_kernel", "rmat20")[0] is None
    assert bench.traffic_for("spmv_bool", 4, "spmv_k4_kernel", "rmat20")[0] is None
    assert bench.traffic_for("spmv_plus", 4, "spmv_chunks_kernel", "rmat20")[0] is None


def test_committed_traffic_entries_are_well_formed():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for key, ent in rec.items():
        assert {"family", "tile_dim", "graph", "kernel", "dram_bytes_per_launch", "kernel_source_sha256",
                "profile"} <= set(ent), key
        assert ent["family"] in bench.FAMILIES
        assert os.path.exists(os.path.join(ROOT, ent["profile"])), ent["profile"]
        assert ent["dram_bytes_per_launch"] > 0


def test_workload_names_the_ids(monkeypatch):
    assert "unpermuted ids" in bench.workload_desc(10, 20)["workload"]
    monkeypatch.setattr(bench, "PERMUTE", 2)
    assert "ids permuted (seed 2)" in bench.workload_desc(10, 20)["workload"]
    assert bench.traffic_key(None) == f"rmat{bench.SCALE}" and bench.traffic_key(2) == f"rmat{bench.SCALE}_perm2"
