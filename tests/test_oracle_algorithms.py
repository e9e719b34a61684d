"""Pins for the oracle's SpGEMM (Table 3), graph algorithms (Sec. V) and
sampling profile (Alg. 1): brute force, closed forms and independent library
routines (scipy.sparse.csgraph), never the oracle's own code path.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import oracle
from paper_2201_08560_gb300 import graphs


def _sp(g):
    return sp.csr_matrix((np.ones(g.nnz), g.colind, g.rowptr), shape=(g.n, g.n))


# ---------------------------------------------------------------- SpGEMM ---

@pytest.mark.parametrize("n,da,db,seed", [(1, 1.0, 1.0, 0), (9, 0.3, 0.2, 1), (40, 0.08, 0.1, 2),
                                          (64, 0.05, 0.05, 3)])
def test_spgemm_bool_and_masked_count(n, da, db, seed):
    A = graphs.random_directed(n, da, seed)
    B = graphs.random_directed(n, db, seed + 50)
    M = graphs.random_directed(n, 0.3, seed + 99)
    a, b, m = graphs.to_dense(A), graphs.to_dense(B), graphs.to_dense(M)
    C = oracle.spgemm_bool(A, B)
    np.testing.assert_array_equal(graphs.to_dense(C), (a @ b > 0).astype(np.int64))
    # sum over M of (A B^T): a transposed operand changes the value on asymmetric inputs
    assert oracle.masked_count(A, B, M) == int((m * (a @ b.T)).sum())


@pytest.mark.parametrize("g", [graphs.complete(7), graphs.random_symmetric(60, 0.2, 5),
                               graphs.mycielski(6), graphs.grid2d(9, 7), graphs.rmat(8, 8, seed=3)])
def test_triangle_count_trace(g):
    a = graphs.to_dense(g)
    assert oracle.triangle_count(g) == int(np.trace(a @ a @ a)) // 6
    # TC = sum(L .* (L L^T)) with L strictly lower (Sec. V TC) equals the masked count
    L = graphs.from_dense(np.tril(a, -1))
    assert oracle.masked_count(L, L, L) == oracle.triangle_count(g)


@pytest.mark.parametrize("n", [3, 4, 10, 25])
def test_triangles_complete_graph(n):
    assert oracle.triangle_count(graphs.complete(n)) == math.comb(n, 3)


@pytest.mark.parametrize("k", [3, 5, 8])
def test_mycielski_triangle_free_and_connected(k):
    g = graphs.mycielski(k)
    assert g.n == 3 * 2 ** (k - 2) - 1
    assert oracle.triangle_count(g) == 0
    assert set(oracle.cc(g).tolist()) == {0}


# -------------------------------------------------------------------- BFS ---

def test_bfs_closed_forms():
    n = 50
    for s in (0, 17, 49):
        np.testing.assert_array_equal(oracle.bfs(graphs.path(n), s), np.abs(np.arange(n) - s))
    lv = oracle.bfs(graphs.complete(12), 4)
    assert lv[4] == 0 and (np.delete(lv, 4) == 1).all()
    R, C = 13, 9
    lv = oracle.bfs(graphs.grid2d(R, C), 0)
    rr, cc = np.divmod(np.arange(R * C), C)
    np.testing.assert_array_equal(lv, rr + cc)
    u = graphs.disjoint_union(graphs.path(4), graphs.cycle(5))
    np.testing.assert_array_equal(oracle.bfs(u, 0), [0, 1, 2, 3, -1, -1, -1, -1, -1])


def test_bfs_matches_scipy():
    g = graphs.rmat(10, 8, seed=4)
    for s in graphs.sources(g, 4, seed=1):
        d = csgraph.shortest_path(_sp(g), method="D", unweighted=True, indices=int(s))
        expect = np.where(np.isinf(d), -1, d).astype(np.int32)
        np.testing.assert_array_equal(oracle.bfs(g, int(s)), expect)


# ------------------------------------------------------------------- SSSP ---

def test_sssp_unit_weights_grid_is_manhattan():
    R, C = 11, 8
    g = graphs.grid2d(R, C)
    rr, cc = np.divmod(np.arange(R * C), C)
    np.testing.assert_array_equal(oracle.sssp(g, 0), (rr + cc).astype(np.float64))
    # unit-weight SSSP equals BFS levels (min-plus with w = 1)
    r = graphs.rmat(9, 8, seed=2)
    lv = oracle.bfs(r, 0).astype(np.float64)
    lv[lv < 0] = np.inf
    np.testing.assert_array_equal(oracle.sssp(r, 0), lv)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_sssp_matches_floyd_warshall(seed):
    g = graphs.random_symmetric(60, 0.08, seed)
    w = graphs.symmetric_weights(g, seed + 3, grid=None)
    m = sp.csr_matrix((w.astype(np.float64), g.colind, g.rowptr), shape=(g.n, g.n))
    fw = csgraph.floyd_warshall(m, directed=True)
    for s in (0, 7, 59):
        np.testing.assert_allclose(oracle.sssp(g, s, w), fw[s], rtol=1e-12)


# --------------------------------------------------------------------- PR ---

@pytest.mark.parametrize("g", [graphs.cycle(17), graphs.torus2d(5, 6), graphs.complete(9)])
def test_pagerank_regular_graph_is_uniform(g):
    for it in (1, 5, 20):
        np.testing.assert_allclose(oracle.pagerank(g, 0.85, it), np.full(g.n, 1.0 / g.n), rtol=1e-14)


def test_pagerank_star_closed_form():
    """Star with centre c and m leaves: c' = (1-d)/n + d*m*l, l' = (1-d)/n + d*c/m."""
    n, d = 11, 0.85
    m = n - 1
    c, l = 1.0 / n, 1.0 / n
    for it in range(1, 15):
        c, l = (1 - d) / n + d * m * l, (1 - d) / n + d * c / m
        x = oracle.pagerank(graphs.star(n), d, it)
        np.testing.assert_allclose(x[0], c, rtol=1e-14)
        np.testing.assert_allclose(x[1:], l, rtol=1e-14)


def test_pagerank_mass_and_dense_power_iteration():
    g = graphs.random_symmetric(80, 0.1, 3)
    a = graphs.to_dense(g).astype(np.float64)
    deg = a.sum(axis=0)
    assert (deg > 0).all()  # no dangling vertices: the total mass stays 1
    x = np.full(g.n, 1.0 / g.n)
    tele = np.random.default_rng(1).random(g.n)
    tele /= tele.sum()
    xt = x.copy()
    for _ in range(30):
        x = 0.15 / g.n + 0.85 * a @ (x / deg)
        xt = 0.15 * tele + 0.85 * a @ (xt / deg)
    np.testing.assert_allclose(oracle.pagerank(g, 0.85, 30), x, rtol=1e-12)
    np.testing.assert_allclose(oracle.pagerank(g, 0.85, 30).sum(), 1.0, rtol=1e-12)
    np.testing.assert_allclose(oracle.pagerank(g, 0.85, 30, tele), xt, rtol=1e-12)


def test_pagerank_dangling_vertices_pass_nothing():
    # directed: 0 -> 1 only (entry (1, 0)); vertex 1 has no out-edges
    g = graphs.from_dense(np.array([[0, 0], [1, 0]]))
    x = oracle.pagerank(g, 0.5, 1)
    np.testing.assert_allclose(x, [0.25, 0.25 + 0.5 * 0.5])


# --------------------------------------------------------------------- CC ---

def test_cc_components():
    parts = [graphs.path(3), graphs.complete(4), graphs.cycle(5), graphs.star(6), graphs.path(1)]
    u = graphs.disjoint_union(*parts)
    lab = oracle.cc(u)
    offs = np.cumsum([0] + [p.n for p in parts])
    expect = np.concatenate([np.full(p.n, o) for p, o in zip(parts, offs[:-1])])
    np.testing.assert_array_equal(lab, expect)


@pytest.mark.parametrize("seed", [0, 5])
def test_cc_matches_scipy(seed):
    g = graphs.permute(graphs.rmat(11, 2, seed=seed), seed + 1)
    ncomp, comp = csgraph.connected_components(_sp(g), directed=False)
    lab = oracle.cc(g)
    assert len(set(lab.tolist())) == ncomp
    # label = minimum vertex id of the component
    for c in range(ncomp):
        members = np.nonzero(comp == c)[0]
        assert (lab[members] == members.min()).all()


# ------------------------------------------------------- sampling profile ---

@pytest.mark.parametrize("g", [graphs.rmat(9, 8, seed=1), graphs.grid2d(16, 16), graphs.mycielski(8)])
def test_sample_profile_full_sample_is_exact(g):
    """With every row sampled once and n divisible by 32, the Alg. 1 estimate is the exact size ratio."""
    assert g.n % 32 == 0 or g.name.startswith("mycielski")
    est, th = oracle.sample_profile(g, np.arange(g.n, dtype=np.int32))
    csr_bytes = 4 * (g.n + 1) + 8 * g.nnz
    for q, k in enumerate(oracle.KS):
        trp, tci, tiles = oracle.b2sr(g, k)
        if g.n % k == 0:
            assert th[q] == pytest.approx(len(tci), rel=1e-12)
            assert est[q] == pytest.approx(oracle.b2sr_bytes(g.n, k, len(tci)) / csr_bytes, rel=1e-12)


# ------------------------------------------------------------ orientation ---

def test_directed_orientation_follows_columns():
    """Entry (i, j) is the edge j -> i, the direction y = A x moves values (Sec. V PR
    uses the column-stochastic matrix): a chain with A[i+1, i] = 1 is walked forward."""
    n = 7
    a = np.zeros((n, n), dtype=np.int64)
    for i in range(n - 1):
        a[i + 1, i] = 1
    fwd = graphs.from_dense(a)
    np.testing.assert_array_equal(oracle.bfs(fwd, 0), np.arange(n))
    np.testing.assert_array_equal(oracle.sssp(fwd, 0), np.arange(n, dtype=np.float64))
    back = graphs.from_dense(a.T)
    assert (oracle.bfs(back, 0)[1:] == -1).all()
    # one SpMV step moves a value from j to i: y = A e_0 reaches vertex 1
    e0 = np.zeros(n)
    e0[0] = 1.0
    np.testing.assert_array_equal(oracle.spmv_plus(fwd, e0), a @ e0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_directed_bfs_sssp_match_scipy_on_transpose(seed):
    g = graphs.random_directed(90, 0.04, seed, self_loops=False)
    w = np.random.default_rng(seed).uniform(0.5, 3.0, g.nnz).astype(np.float32)
    At = sp.csr_matrix((w.astype(np.float64), g.colind, g.rowptr), shape=(g.n, g.n)).T.tocsr()
    for s in (0, 13, 89):
        d = csgraph.shortest_path(At, method="D", directed=True, indices=s)
        np.testing.assert_allclose(oracle.sssp(g, s, w), d, rtol=1e-12)
        hops = csgraph.shortest_path(At, method="D", directed=True, unweighted=True, indices=s)
        np.testing.assert_array_equal(oracle.bfs(g, s), np.where(np.isinf(hops), -1, hops).astype(np.int32))


def test_fullsize_tc_golden_input_is_reproduced():
    """The stored full-size triangle count belongs to the graph the seeded
    generator makes on this machine (same sizes and CSR digest)."""
    import hashlib
    import json
    import os
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "fullsize_tc.json")))
    g = graphs.rmat(18, 32, seed=2)
    h = hashlib.sha256()
    h.update(g.rowptr.astype("<i8").tobytes())
    h.update(g.colind.astype("<i4").tobytes())
    assert (g.n, len(g.colind), h.hexdigest()) == (gold["n"], gold["nnz"], gold["csr_sha256"])
