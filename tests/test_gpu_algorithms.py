"""GPU parity: SpGEMM (Table 3 and the Boolean product) and the Sec. V graph
algorithms (BFS, multi-source BFS, SSSP, PageRank, CC, TC) against the oracle.
Levels, labels and counts are bit-exact; PageRank and continuous-weight SSSP
are within 1e-5 relative error of the fp64 oracle."""
import itertools
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import GRAPH_IDS, csr_dev, small_graphs, to_dev, to_np

pytestmark = pytest.mark.gpu

KS = [4, 8, 16, 32]


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


def mat(B, g, k):
    rp, ci = csr_dev(g)
    return B.b2sr_from_csr(g.n, rp, ci, k)


# ---------------------------------------------------------------- SpGEMM ---

@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("n,da,db,seed", [(1, 1.0, 1.0, 0), (77, 0.08, 0.1, 1), (300, 0.02, 0.03, 2)])
def test_masked_count_asymmetric(B, k, n, da, db, seed):
    A = graphs.random_directed(n, da, seed)
    Bm = graphs.random_directed(n, db, seed + 50)
    M = graphs.random_directed(n, 0.3, seed + 99)
    with mat(B, A, k) as a, mat(B, Bm, k) as b, mat(B, M, k) as mm:
        got = int(B.b2sr_spgemm_masked_count(a, b, mm).item())
    assert got == oracle.masked_count(A, Bm, M)


def _tile_pairs(A, Bm, M, k):
    """Work of the masked count from the oracle's B2SR arrays: over every mask
    tile (I, J), its set bits times the tile-columns K stored in both A's
    tile-row I and B's tile-row J."""
    def rows(g):
        trp, tci, tiles = oracle.b2sr(g, k)
        return [set(tci[trp[i]:trp[i + 1]].tolist()) for i in range(len(trp) - 1)], trp, tci, tiles
    ra, _, _, _ = rows(A)
    rb, _, _, _ = rows(Bm)
    _, mrp, mci, mtiles = rows(M)
    total = 0
    for i in range(len(mrp) - 1):
        for t in range(mrp[i], mrp[i + 1]):
            bits = sum(bin(int(w)).count("1") for w in np.atleast_1d(mtiles[t]))
            total += bits * len(ra[i] & rb[int(mci[t])])
    return total


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("n,da,db,seed", [(1, 1.0, 1.0, 0), (77, 0.08, 0.1, 1), (300, 0.02, 0.03, 2)])
def test_masked_count_work(B, k, n, da, db, seed):
    """The count with its work report equals the plain count, and the reported
    AND-popc operations equal the tile-level work computed from the oracle's
    tile arrays."""
    A = graphs.random_directed(n, da, seed)
    Bm = graphs.random_directed(n, db, seed + 50)
    M = graphs.random_directed(n, 0.3, seed + 99)
    with mat(B, A, k) as a, mat(B, Bm, k) as b, mat(B, M, k) as mm:
        cnt, pairs = B.b2sr_spgemm_masked_count_work(a, b, mm)
    assert int(cnt.item()) == oracle.masked_count(A, Bm, M)
    assert int(pairs.item()) == _tile_pairs(A, Bm, M, k)


def _hub_with_path(n):
    """Vertex 0 joined to every other vertex, and the others joined in a path:
    n - 2 triangles (0, i, i+1), all through one hub row."""
    i = np.arange(1, n, dtype=np.int64)
    src = np.concatenate([np.zeros(n - 1, np.int64), i[:-1]])
    dst = np.concatenate([i, i[1:]])
    return graphs.from_edges(n, src, dst)


@pytest.mark.parametrize("k", [4, 8])
def test_masked_count_long_row(B, k):
    """A mask tile-row whose A row has more tiles than the staged list holds
    (a hub with 199,999 neighbours): positions are then searched in global
    memory."""
    g = _hub_with_path(200000)
    with mat(B, g, k) as m:
        assert int(B.b2sr_spgemm_masked_count(m, m, m).item()) == oracle.masked_count(g, g, g)
        assert int(B.b2sr_tc(m).item()) == 200000 - 2


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", [0, 1, 2, 3, 4, 6, 7, 8], ids=["rmat12", "rmat11perm", "star20k", "grid37x41",
                                                               "gaps", "n1", "empty45", "mycielski9"])
def test_triangle_count(B, k, gi):
    g = small_graphs()[gi]
    with mat(B, g, k) as m:
        assert int(B.b2sr_tc(m).item()) == oracle.triangle_count(g)


@pytest.mark.parametrize("n", [5, 33, 70])
def test_triangle_count_complete(B, n):
    g = graphs.complete(n)
    for k in KS:
        with mat(B, g, k) as m:
            assert int(B.b2sr_tc(m).item()) == math.comb(n, 3)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("n,da,db,seed", [(1, 1.0, 1.0, 0), (90, 0.05, 0.05, 1), (257, 0.01, 0.02, 2)])
def test_spgemm_bool(B, k, n, da, db, seed):
    A = graphs.random_directed(n, da, seed)
    Bm = graphs.random_directed(n, db, seed + 7)
    C = oracle.spgemm_bool(A, Bm)
    with mat(B, A, k) as a, mat(B, Bm, k) as b, B.b2sr_spgemm_bool(a, b) as c:
        rp, ci = B.b2sr_to_csr(c)
        np.testing.assert_array_equal(to_np(rp), C.rowptr)
        np.testing.assert_array_equal(to_np(ci), C.colind)
        trp, tci, tiles = oracle.b2sr(C, k)
        assert c.n_tiles == len(tci)


def test_spgemm_bool_rmat(B):
    g = graphs.rmat(10, 8, seed=2)
    C = oracle.spgemm_bool(g, g)
    for k in KS:
        with mat(B, g, k) as a, B.b2sr_spgemm_bool(a, a) as c:
            rp, ci = B.b2sr_to_csr(c)
            np.testing.assert_array_equal(to_np(ci), C.colind)


# ------------------------------------------------------------------- BFS ---

@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
def test_bfs(B, k, gi):
    g = small_graphs()[gi]
    gc = oracle.canonicalize(g)
    srcs = [0, g.n - 1, g.n // 2]
    with mat(B, g, k) as m:
        for s in srcs:
            np.testing.assert_array_equal(to_np(B.b2sr_bfs(m, s)), oracle.bfs(gc, s))


def test_bfs_closed_forms(B):
    for k in KS:
        with mat(B, graphs.path(300), k) as m:
            np.testing.assert_array_equal(to_np(B.b2sr_bfs(m, 17)), np.abs(np.arange(300) - 17))
        R, C = 45, 38
        with mat(B, graphs.grid2d(R, C), k) as m:
            rr, cc = np.divmod(np.arange(R * C), C)
            np.testing.assert_array_equal(to_np(B.b2sr_bfs(m, 0)), rr + cc)


def test_bfs_errors(B):
    g = graphs.path(50)
    with mat(B, g, 8) as m:
        with pytest.raises(B.B2SRError) as e:
            B.b2sr_bfs(m, 50)
        assert e.value.status == 1
        with pytest.raises(B.B2SRError) as e:
            B.b2sr_bfs(m, 0, max_iters=10)   # the path needs 49 levels
        assert e.value.status == 5


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", [0, 1, 3, 4, 5], ids=["rmat12", "rmat11perm", "grid37x41", "gaps", "directed300"])
def test_bfs_multi(B, k, gi):
    g = small_graphs()[gi]
    gc = oracle.canonicalize(g)
    srcs = list(graphs.sources(g, 64, seed=gi)) if gi != 4 else list(range(0, g.n, max(1, g.n // 40)))[:64]
    with mat(B, g, k) as m:
        lv = to_np(B.b2sr_bfs_multi(m, srcs))
        for s_i, s in enumerate(srcs):
            np.testing.assert_array_equal(lv[s_i], oracle.bfs(gc, int(s)))
        # smaller batches give the same rows: 3 and 32 sources run on 32-lane
        # words, 33 and more on 64-lane words
        for cnt in (3, 32, 33):
            if cnt <= len(srcs):
                np.testing.assert_array_equal(to_np(B.b2sr_bfs_multi(m, srcs[:cnt])), lv[:cnt])


# ------------------------------------------------------------------ SSSP ---

@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", [0, 3, 4, 5], ids=["rmat12", "grid37x41", "gaps", "directed300"])
def test_sssp(B, k, gi):
    g = oracle.canonicalize(small_graphs()[gi])
    rng = np.random.default_rng(gi)
    w_grid = (1 + rng.integers(0, 99 * 16, g.colind.size) / 16).astype(np.float32)
    w_cont = rng.uniform(1.0, 100.0, g.colind.size).astype(np.float32)
    rp, ci = to_dev(g.rowptr), to_dev(g.colind)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        # unit weights: distances equal BFS levels
        d = to_np(B.b2sr_sssp(m, 0))
        lv = oracle.bfs(g, 0).astype(np.float64)
        lv[lv < 0] = np.inf
        np.testing.assert_array_equal(d.astype(np.float64), lv)
        for w, exact in ((w_grid, True), (w_cont, False)):
            wb = B.b2sr_weights_from_csr(m, rp, ci, to_dev(w))
            d = to_np(B.b2sr_sssp(m, 1, wb)).astype(np.float64)
            ref = oracle.sssp(g, 1, w)
            if exact:
                np.testing.assert_array_equal(d, ref)
            else:
                fin = np.isfinite(ref)
                assert (np.isfinite(d) == fin).all()
                np.testing.assert_allclose(d[fin], ref[fin], rtol=1e-5)


# -------------------------------------------------------------------- PR ---

@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", [0, 1, 2, 3, 4, 5, 8], ids=["rmat12", "rmat11perm", "star20k", "grid37x41", "gaps",
                                                            "directed300", "mycielski9"])
def test_pagerank(B, k, gi):
    g = oracle.canonicalize(small_graphs()[gi])
    rp, ci = to_dev(g.rowptr), to_dev(g.colind)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        for iters in (1, 20, 50):
            pr = to_np(B.b2sr_pagerank(m, 0.85, iters)).astype(np.float64)
            ref = oracle.pagerank(g, 0.85, iters)
            np.testing.assert_allclose(pr, ref, rtol=1e-5, atol=0)
        tele = np.random.default_rng(gi).random(g.n)
        tele /= tele.sum()
        pr = to_np(B.b2sr_pagerank(m, 0.85, 20, to_dev(tele.astype(np.float32)))).astype(np.float64)
        ref = oracle.pagerank(g, 0.85, 20, tele.astype(np.float32).astype(np.float64))
        np.testing.assert_allclose(pr, ref, rtol=1e-5, atol=0)


def test_pagerank_closed_forms(B):
    for g in (graphs.cycle(1000), graphs.torus2d(30, 40)):
        for k in KS:
            with mat(B, g, k) as m:
                np.testing.assert_allclose(to_np(B.b2sr_pagerank(m, 0.85, 30)), 1.0 / g.n, rtol=1e-6)


# -------------------------------------------------------------------- CC ---

@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", [0, 1, 2, 3, 4, 6, 7, 8], ids=["rmat12", "rmat11perm", "star20k", "grid37x41",
                                                               "gaps", "n1", "empty45", "mycielski9"])
def test_cc(B, k, gi):
    g = small_graphs()[gi]
    with mat(B, g, k) as m:
        np.testing.assert_array_equal(to_np(B.b2sr_cc(m)), oracle.cc(oracle.canonicalize(g)))


def test_cc_disjoint_unions(B):
    parts = [graphs.path(300), graphs.complete(9), graphs.cycle(41), graphs.star(77), graphs.path(1),
             graphs.grid2d(20, 30)]
    u = graphs.permute(graphs.disjoint_union(*parts), seed=3)
    for k in KS:
        with mat(B, u, k) as m:
            lab = to_np(B.b2sr_cc(m))
            np.testing.assert_array_equal(lab, oracle.cc(u))
            assert len(set(lab.tolist())) == len(parts)


def transposed(g, w):
    """A^T of a canonical CSR, with each entry's weight carried over."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.rowptr))
    order = np.lexsort((rows, g.colind.astype(np.int64)))
    rp = np.zeros(g.n + 1, dtype=np.int32)
    np.cumsum(np.bincount(g.colind, minlength=g.n), out=rp[1:])
    return graphs.CSR(g.n, rp, rows[order].astype(np.int32)), w[order]


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
def test_sssp_push(B, k, gi):
    """Push SSSP on the transpose: unit weights give BFS levels, lattice
    weights the oracle's distances bit for bit, continuous weights exactly the
    pull rounds' result (both reach the same least fixed point of the fp32
    relaxation)."""
    g = oracle.canonicalize(small_graphs()[gi])
    rng = np.random.default_rng(gi + 100)
    w_grid = (1 + rng.integers(0, 99 * 16, g.colind.size) / 16).astype(np.float32)
    w_cont = rng.uniform(1.0, 100.0, g.colind.size).astype(np.float32)
    rp, ci = to_dev(g.rowptr), to_dev(g.colind)
    src = min(1, g.n - 1)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        gT, _ = transposed(g, w_grid)
        rpT, ciT = to_dev(gT.rowptr), to_dev(gT.colind)
        with B.b2sr_from_csr(g.n, rpT, ciT, k) as mT:
            d = to_np(B.b2sr_sssp_push(mT, 0))
            lv = oracle.bfs(g, 0).astype(np.float64)
            lv[lv < 0] = np.inf
            np.testing.assert_array_equal(d.astype(np.float64), lv)
            np.testing.assert_array_equal(to_np(B.b2sr_sssp_push(mT, 0, delta=1.0)).astype(np.float64), lv)
            for (w, exact), delta in itertools.product(((w_grid, True), (w_cont, False)), (0.0, 7.0, 100.0)):
                _, wT = transposed(g, w)
                wbT = B.b2sr_weights_from_csr(mT, rpT, ciT, to_dev(wT))
                d = to_np(B.b2sr_sssp_push(mT, src, wbT, delta=delta))
                if exact:
                    np.testing.assert_array_equal(d.astype(np.float64), oracle.sssp(g, src, w))
                else:
                    wb = B.b2sr_weights_from_csr(m, rp, ci, to_dev(w))
                    np.testing.assert_array_equal(d.view(np.uint32), to_np(B.b2sr_sssp(m, src, wb)).view(np.uint32))


@pytest.mark.parametrize("k", KS)
def test_sssp_push_rounds_on_a_path(B, k):
    """Unit weights on a path from one end: one round per hop, plus the round
    that finds nothing left to improve."""
    g = graphs.path(203)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        d = to_np(B.b2sr_sssp_push(m, 0))
        np.testing.assert_array_equal(d, np.arange(g.n, dtype=np.float32))
        assert B.b2sr_sssp_push_rounds() == g.n
        # one active vertex, hence one active tile-row, in each of the n rounds
        assert B.b2sr_sssp_push_rounds(with_rows=True) == (g.n, g.n)
        with pytest.raises(B.B2SRError):
            B.b2sr_sssp_push(m, 0, max_iters=5)
        assert B.b2sr_sssp_push_rounds() == 0


@pytest.mark.parametrize("k", KS)
def test_sssp_push_far_set(B, k):
    """Thresholds from below the lightest edge to past the longest path: the
    far set holds most of the graph for the small ones, none of it for the
    large one; every delta gives the oracle's distances."""
    g = graphs.grid2d(45, 38)
    w = graphs.symmetric_weights(g, 5)
    rp, ci = csr_dev(g)
    want = oracle.sssp(g, 7, w)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        wb = B.b2sr_weights_from_csr(m, rp, ci, to_dev(w))
        rounds = {}
        for delta in (0.0, 0.75, 3.0, 40.0, 1e6):
            d = to_np(B.b2sr_sssp_push(m, 7, wb, delta=delta))
            np.testing.assert_array_equal(d.astype(np.float64), want)
            rounds[delta] = B.b2sr_sssp_push_rounds()
        # narrow buckets: more raises of the threshold, fewer rounds in each
        assert rounds[0.75] > rounds[40.0]
        assert max(rounds.values()) <= 4 * g.n + 4


def test_sssp_push_symmetric_uses_own_handle(B):
    g = graphs.grid2d(60, 70)
    w = graphs.symmetric_weights(g, 3)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        wb = B.b2sr_weights_from_csr(m, rp, ci, to_dev(w))
        for delta in (0.0, 50.0):
            d = to_np(B.b2sr_sssp_push(m, 0, wb, delta=delta))
            np.testing.assert_array_equal(d.astype(np.float64), oracle.sssp(g, 0, w))
            np.testing.assert_array_equal(d, to_np(B.b2sr_sssp(m, 0, wb)))
            with pytest.raises(B.B2SRError):
                B.b2sr_sssp_push(m, 0, wb, delta=delta, max_iters=5)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
def test_bfs_diropt(B, k, gi):
    """Direction-optimising BFS equals the oracle's levels (and b2sr_bfs's),
    with the transpose given explicitly and, for symmetric graphs, implied."""
    g = oracle.canonicalize(small_graphs()[gi])
    rp, ci = to_dev(g.rowptr), to_dev(g.colind)
    gT, _ = transposed(g, np.zeros(g.colind.size, np.float32))
    with B.b2sr_from_csr(g.n, rp, ci, k) as m, \
            B.b2sr_from_csr(g.n, to_dev(gT.rowptr), to_dev(gT.colind), 4 if k != 4 else 8) as mT:
        for src in sorted({0, g.n // 2, g.n - 1}):
            ref = oracle.bfs(g, src)
            np.testing.assert_array_equal(to_np(B.b2sr_bfs_diropt(m, src, mT)), ref)
            symmetric = np.array_equal(gT.rowptr, g.rowptr) and np.array_equal(gT.colind, g.colind)
            if symmetric:
                np.testing.assert_array_equal(to_np(B.b2sr_bfs_diropt(m, src)), ref)


def test_bfs_diropt_switches_direction(B):
    """On R-MAT the search pushes, pulls through the dense middle levels and
    pushes again; on a long path it pushes throughout.  Either way: the oracle's
    levels, and the level cap still applies."""
    for g in (graphs.rmat(14, 16, seed=3), graphs.path(3000), graphs.grid2d(90, 70)):
        rp, ci = csr_dev(g)
        with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
            np.testing.assert_array_equal(to_np(B.b2sr_bfs_diropt(m, 0)), oracle.bfs(g, 0))
    g = graphs.path(100)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        with pytest.raises(B.B2SRError):
            B.b2sr_bfs_diropt(m, 0, max_iters=10)


# ---------------------------------------------------------------------------
# B2SR of the transpose (Sec. III-A CSR -> CSC of the tile index, Sec. III-B
# transposed tile packing)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
def test_transpose_arrays_and_vxm(B, k, gi):
    g = oracle.canonicalize(small_graphs()[gi])
    gt, _ = transposed(g, np.zeros(g.colind.size, np.float32))
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m, B.b2sr_transpose(m) as mt:
        assert (mt.n, mt.tile_dim, mt.nnz) == (m.n, m.tile_dim, m.nnz)
        trp, tci, tiles = B.b2sr_export(mt)
        otrp, otci, otiles = oracle.b2sr(gt, k)
        assert mt.n_tiles == len(otci)
        np.testing.assert_array_equal(to_np(trp), otrp)
        ob = otiles.reshape(-1).view(np.uint8)
        np.testing.assert_array_equal(to_np(tci)[: len(otci)], otci)
        np.testing.assert_array_equal(to_np(tiles)[: ob.size], ob)
        # transposing twice gives the original arrays back
        with B.b2sr_transpose(mt) as mtt:
            a, b = B.b2sr_export(mtt), B.b2sr_export(m)
            nb = ob.size
            assert torch.equal(a[0], b[0])
            assert torch.equal(a[1][: m.n_tiles], b[1][: m.n_tiles])
            assert torch.equal(a[2][:nb], b[2][:nb])
        # vxm: x^T A = A^T x
        xb = graphs.random_bits(g.n, 0.3, seed=gi + 2)
        y = torch.empty(max(B.bitset_words(g.n), 1), dtype=torch.int32, device="cuda")
        B.b2sr_spmv(mt, B.BOOL_OR_AND, B.VEC_BITS, to_dev(xb), B.VEC_BITS, y)
        np.testing.assert_array_equal(to_np(y, np.uint32)[: B.bitset_words(g.n)], oracle.spmv_bool(gt, xb))
        x = (np.random.default_rng(gi).integers(0, 1000, g.n) / 4).astype(np.float32)   # exact sums
        yf = torch.empty(max(g.n, 1), dtype=torch.float32, device="cuda")
        B.b2sr_spmv(mt, B.PLUS_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, yf)
        np.testing.assert_array_equal(to_np(yf)[: g.n], oracle.spmv_plus(gt, x.astype(np.float64)).astype(np.float32))


@pytest.mark.parametrize("k", [4, 8, 32])
def test_push_drivers_on_device_transpose(B, k):
    """Directed graphs: the push drivers read A^T made on the device."""
    g = oracle.canonicalize(graphs.random_directed(700, 0.01, seed=5))
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m, B.b2sr_transpose(m) as mt:
        for s in (0, 17, 350):
            np.testing.assert_array_equal(to_np(B.b2sr_bfs_diropt(m, s, mt)), oracle.bfs(g, s))
            np.testing.assert_array_equal(to_np(B.b2sr_sssp_push(mt, s)), oracle.sssp(g, s).astype(np.float32))
