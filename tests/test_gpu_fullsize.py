"""GPU parity at the benchmark sizes, through the same entry points and
launch configuration the benchmark times:

  * R-MAT scale 20 ef16 (the main workload, at k = 4 with the direct
    schedule as the benchmark runs it, and at k = 8 with the default one): the
    B2SR arrays, the Boolean, plus-times and int-min SpMVs, PageRank (50
    iterations) and CC against the oracle in full; the 16-source batched BFS
    on three sampled sources in full; MIS and colouring with a random
    priority permutation in full;
  * the 4096 x 4096 grid with lattice weights: push SSSP from the corner, in
    full and bit-exact (every path sum is exact in fp32);
  * R-MAT scale 18 ef32: the triangle count against the oracle's count stored
    in tests/golden/fullsize_tc.json (written by make_fullsize_golden.py);
  * R-MAT scale 22 ef16: the 64-source BFS on two sampled sources in full.

Tolerances as in the small-size tests: bit-exact for bits, levels, labels
and counts; 1e-5 relative for fp32 PageRank and plus-times."""
import hashlib
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import csr_dev, to_dev, to_np

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
RTOL = 1e-5


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def rmat20_graph():
    return graphs.rmat(20, 16, seed=1)


@pytest.fixture(scope="module", params=[(4, 2), (8, 0)], ids=["k4-direct", "k8"])
def rmat20(B, rmat20_graph, request):
    g = rmat20_graph
    k, sched = request.param
    rp, ci = csr_dev(g)
    m = B.b2sr_from_csr(g.n, rp, ci, k)
    B.b2sr_set_schedule(m, sched)
    yield g, m
    m.close()


def test_rmat20_b2sr_arrays(B, rmat20):
    g, m = rmat20
    trp, tci, tiles = B.b2sr_export(m)
    otrp, otci, otiles = oracle.b2sr(g, m.tile_dim)
    assert m.n_tiles == len(otci) and m.nnz == len(g.colind)
    np.testing.assert_array_equal(to_np(trp), otrp)
    np.testing.assert_array_equal(to_np(tci), otci)
    np.testing.assert_array_equal(to_np(tiles), otiles.reshape(-1).view(np.uint8))


def test_rmat20_spmv(B, rmat20):
    g, m = rmat20
    xb = graphs.random_bits(g.n, 0.05, seed=3)          # the benchmark's vector
    y = torch.empty(B.bitset_words(g.n), dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, to_dev(xb), B.VEC_BITS, y)
    np.testing.assert_array_equal(to_np(y, np.uint32), oracle.spmv_bool(g, xb))
    x = np.random.default_rng(4).random(g.n).astype(np.float32)
    yf = torch.empty(g.n, dtype=torch.float32, device="cuda")
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, yf)
    np.testing.assert_allclose(to_np(yf).astype(np.float64), oracle.spmv_plus(g, x.astype(np.float64)),
                               rtol=RTOL, atol=0)
    xi = np.random.default_rng(5).integers(0, 1 << 30, g.n).astype(np.int32)
    yi = torch.empty(g.n, dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_I32, to_dev(xi), B.VEC_I32, yi)
    np.testing.assert_array_equal(to_np(yi), oracle.spmv_min_i32(g, xi))


def test_rmat20_bfs16_sampled(B, rmat20):
    g, m = rmat20
    srcs = graphs.sources(g, 16, seed=7)                 # the benchmark's sources
    lv = to_np(B.b2sr_bfs_multi(m, [int(s) for s in srcs]))
    for i in (0, 7, 15):
        np.testing.assert_array_equal(lv[i], oracle.bfs(g, int(srcs[i])), err_msg=f"source {i}")


def test_rmat20_pagerank50(B, rmat20):
    g, m = rmat20
    pr = to_np(B.b2sr_pagerank(m, 0.85, 50)).astype(np.float64)
    np.testing.assert_allclose(pr, oracle.pagerank(g, 0.85, 50), rtol=RTOL, atol=0)


def test_rmat20_cc(B, rmat20):
    g, m = rmat20
    np.testing.assert_array_equal(to_np(B.b2sr_cc(m)), oracle.cc(g))


def test_rmat20_mis_and_colouring(B, rmat20):
    g, m = rmat20
    pr = np.random.default_rng(31).permutation(g.n).astype(np.float32) + 1.0   # the benchmark's priorities
    p = torch.from_numpy(pr).cuda()
    np.testing.assert_array_equal(to_np(B.b2sr_mis(m, p)), oracle.mis_greedy(g, pr.astype(np.float64)))
    ref = oracle.color_levels(g, pr.astype(np.float64))
    np.testing.assert_array_equal(to_np(B.b2sr_color(m, p, method=B.COLOR_PUSH)), ref)
    np.testing.assert_array_equal(to_np(B.b2sr_color(m, p, method=B.COLOR_MAX_TIMES)), ref)


def test_grid4096_sssp(B):
    g = graphs.grid2d(4096, 4096)
    w = graphs.symmetric_weights(g, 5)                   # the benchmark's weights
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        wb = B.b2sr_weights_from_csr(m, rp, ci, to_dev(w))
        d = to_np(B.b2sr_sssp_push(m, 0, wb, delta=400.0))   # the benchmark's driver and delta
    np.testing.assert_array_equal(d, oracle.sssp(g, 0, w).astype(np.float32))


def test_rmat18_ef32_tc(B):
    gold = json.load(open(os.path.join(HERE, "golden", "fullsize_tc.json")))
    g = graphs.rmat(18, 32, seed=2)
    h = hashlib.sha256()
    h.update(g.rowptr.astype("<i8").tobytes())
    h.update(g.colind.astype("<i4").tobytes())
    assert h.hexdigest() == gold["csr_sha256"]           # the graph the count was made for
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        assert int(B.b2sr_tc(m).item()) == gold["triangles"]


def test_rmat22_bfs64_sampled(B):
    g = graphs.rmat(22, 16, seed=3)
    rng = np.random.default_rng(17)
    cand = np.flatnonzero(np.diff(g.rowptr) > 0)
    srcs = [int(v) for v in cand[rng.integers(0, cand.size, 64)]]
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        lv = B.b2sr_bfs_multi(m, srcs)
        rows = {i: to_np(lv[i]) for i in (0, 63)}
    del lv
    for i, row in rows.items():
        np.testing.assert_array_equal(row, oracle.bfs(g, srcs[i]), err_msg=f"source {i}")
