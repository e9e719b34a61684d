"""GPU parity at the benchmark sizes, through the same entry points and
launch configuration the benchmark times:

  * R-MAT scale 20 ef16, with unpermuted and with randomly permuted ids (the
    two graphs of the benchmark's configuration), each at k = 4 with the
    direct schedule (as the benchmark runs it) and at k = 8 with the default
    one: the B2SR arrays, the Boolean, plus-times and int-min SpMVs, PageRank
    (50 iterations), CC and all 16 lanes of the batched BFS against the oracle
    in full; MIS and colouring with a random priority permutation in full;
  * R-MAT scale 20 unpermuted at k = 16 and 32 (the rest of the tile_dim
    sweep): the Boolean and plus-times SpMVs in full;
  * the 4096 x 4096 grid with lattice weights: push SSSP from the corner, in
    full and bit-exact (every path sum is exact in fp32);
  * R-MAT scale 18 ef32: the triangle count against the oracle's count stored
    in tests/golden/fullsize_tc.json (written by make_fullsize_golden.py);
  * R-MAT scale 22 ef16: the 64-source BFS, 18 lanes spread over the 64
    (including the first two and the last two) in full.

Tolerances as in the small-size tests: bit-exact for bits, levels, labels
and counts; 1e-5 relative for fp32 PageRank and plus-times."""
import functools
import hashlib
import json
import os
from concurrent.futures import ThreadPoolExecutor

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


@functools.lru_cache(maxsize=2)
def rmat20_graph(perm: bool):
    g = graphs.rmat(20, 16, seed=1)
    return graphs.permute(g, 2) if perm else g


@functools.lru_cache(maxsize=64)
def oracle_result(perm: bool, what: str, *args):
    """Oracle results per graph, shared by the tile sizes (each is computed once)."""
    g = rmat20_graph(perm)
    return getattr(oracle, what)(g, *args)


def oracle_bfs_many(g, srcs):
    """The oracle's BFS from several sources, on host threads (each call is independent)."""
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        return list(ex.map(lambda s: oracle.bfs(g, int(s)), srcs))


@pytest.fixture(scope="module", params=[(False, 4, 2), (False, 8, 0), (True, 4, 2), (True, 8, 0)],
                ids=["k4-direct", "k8", "perm-k4-direct", "perm-k8"])
def rmat20(B, request):
    perm, k, sched = request.param
    g = rmat20_graph(perm)
    rp, ci = csr_dev(g)
    m = B.b2sr_from_csr(g.n, rp, ci, k)
    B.b2sr_set_schedule(m, sched)
    yield g, m, perm
    m.close()


def test_rmat20_b2sr_arrays(B, rmat20):
    g, m, perm = rmat20
    trp, tci, tiles = B.b2sr_export(m)
    otrp, otci, otiles = oracle_result(perm, "b2sr", m.tile_dim)
    assert m.n_tiles == len(otci) and m.nnz == len(g.colind)
    np.testing.assert_array_equal(to_np(trp), otrp)
    np.testing.assert_array_equal(to_np(tci), otci)
    np.testing.assert_array_equal(to_np(tiles), otiles.reshape(-1).view(np.uint8))


XB_SEED, XF_SEED, XI_SEED = 3, 4, 5


@functools.lru_cache(maxsize=2)
def _oracle_bool(perm):
    g = rmat20_graph(perm)
    return oracle.spmv_bool(g, graphs.random_bits(g.n, 0.05, seed=XB_SEED))


def _spmvs(B, g, m, perm, int_min=True):
    xb = graphs.random_bits(g.n, 0.05, seed=XB_SEED)    # the benchmark's vector
    y = torch.empty(B.bitset_words(g.n), dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, to_dev(xb), B.VEC_BITS, y)
    np.testing.assert_array_equal(to_np(y, np.uint32), _oracle_bool(perm))
    x = np.random.default_rng(XF_SEED).random(g.n).astype(np.float32)
    yf = torch.empty(g.n, dtype=torch.float32, device="cuda")
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, yf)
    np.testing.assert_allclose(to_np(yf).astype(np.float64), oracle.spmv_plus(g, x.astype(np.float64)),
                               rtol=RTOL, atol=0)
    if int_min:
        xi = np.random.default_rng(XI_SEED).integers(0, 1 << 30, g.n).astype(np.int32)
        yi = torch.empty(g.n, dtype=torch.int32, device="cuda")
        B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_I32, to_dev(xi), B.VEC_I32, yi)
        np.testing.assert_array_equal(to_np(yi), oracle.spmv_min_i32(g, xi))


def test_rmat20_spmv(B, rmat20):
    g, m, perm = rmat20
    _spmvs(B, g, m, perm)


@pytest.mark.parametrize("k", [16, 32])
def test_rmat20_spmv_k16_k32(B, k):
    """The tile_dim sweep's other two sizes on the unpermuted graph."""
    g = rmat20_graph(False)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        for sched in (0, 2):
            B.b2sr_set_schedule(m, sched)
            _spmvs(B, g, m, False, int_min=False)


def test_rmat20_bfs16_all_lanes(B, rmat20):
    g, m, perm = rmat20
    srcs = graphs.sources(g, 16, seed=7)                 # the benchmark's sources
    lv = to_np(B.b2sr_bfs_multi(m, [int(s) for s in srcs]))
    refs = _bfs16(perm, tuple(int(s) for s in srcs))
    for i in range(16):
        np.testing.assert_array_equal(lv[i], refs[i], err_msg=f"source {i}")


@functools.lru_cache(maxsize=2)
def _bfs16(perm, srcs):
    return oracle_bfs_many(rmat20_graph(perm), srcs)


def test_rmat20_pagerank50(B, rmat20):
    g, m, perm = rmat20
    pr = to_np(B.b2sr_pagerank(m, 0.85, 50)).astype(np.float64)
    np.testing.assert_allclose(pr, oracle_result(perm, "pagerank", 0.85, 50), rtol=RTOL, atol=0)


def test_rmat20_cc(B, rmat20):
    g, m, perm = rmat20
    np.testing.assert_array_equal(to_np(B.b2sr_cc(m)), oracle_result(perm, "cc"))


def test_rmat20_mis_and_colouring(B, rmat20):
    g, m, perm = rmat20
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


def test_rmat22_bfs64_lanes(B):
    g = graphs.rmat(22, 16, seed=3)
    rng = np.random.default_rng(17)
    cand = np.flatnonzero(np.diff(g.rowptr) > 0)
    srcs = [int(v) for v in cand[rng.integers(0, cand.size, 64)]]   # the benchmark's sources
    lanes = sorted({0, 1, 62, 63, *range(5, 62, 4)})                 # 18 lanes across the 64
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        lv = B.b2sr_bfs_multi(m, srcs)
        rows = {i: to_np(lv[i]) for i in lanes}
    del lv
    refs = oracle_bfs_many(g, [srcs[i] for i in lanes])
    for i, ref in zip(lanes, refs):
        np.testing.assert_array_equal(rows[i], ref, err_msg=f"source {i}")
