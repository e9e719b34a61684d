"""GPU parity for batched work: many uneven graphs packed block-diagonally in
one B2SR arena (b2sr_from_csr_batch) and BFS from a set of sources
(b2sr_bfs_sources), whose level rounds run as a replayed CUDA graph.  Each
graph's slice of the arena result must equal the oracle's BFS of that graph
alone, bit for bit (Sec. V BFS)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import csr_dev, to_np

pytestmark = pytest.mark.gpu

KS = [4, 8, 16, 32]


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


def uneven_graphs():
    """Forty graphs from 0 to ~4k vertices: R-MAT of several scales, paths
    (deep BFS), stars, grids, random directed graphs, empty and single-vertex."""
    gs = []
    for i in range(10):
        gs.append(graphs.rmat(6 + i % 6, 4 + 2 * (i % 4), seed=100 + i))
    gs += [graphs.path(n) for n in (1, 2, 31, 33, 700)]
    gs += [graphs.star(n) for n in (3, 64, 1000)]
    gs += [graphs.grid2d(r, c) for r, c in ((1, 1), (7, 9), (31, 33), (50, 20))]
    gs += [graphs.random_directed(n, 4.0 / max(n, 1), seed=200 + n) for n in (5, 40, 129, 600, 1500)]
    gs += [graphs.from_edges(n, np.zeros(0, np.int64), np.zeros(0, np.int64)) for n in (0, 1, 17)]
    gs += [graphs.mycielski(k) for k in (4, 7, 9)]
    gs += [graphs.cycle(n) for n in (3, 97, 1024)]
    gs += [graphs.rmat(12, 8, seed=7), graphs.permute(graphs.rmat(11, 16, seed=8), 9)]
    gs += [graphs.complete(40), graphs.torus2d(16, 16)]
    return gs


def arena(B, gs, k):
    csrs = []
    for g in gs:
        rp, ci = csr_dev(g)
        csrs.append((g.n, rp, ci))
    m, bases = B.b2sr_from_csr_batch(csrs, k)
    return m, bases, csrs   # csrs keep the inputs alive until the conversion is done


def test_arena_bases_and_structure(B):
    gs = uneven_graphs()
    m, bases, _ = arena(B, gs, 8)
    with m:
        assert bases[0] == 0
        for g, b0, b1 in zip(gs, bases[:-1], bases[1:]):
            assert b0 % 32 == 0 and b1 - b0 == -(-g.n // 32) * 32
        assert m.n == bases[-1]
        rp, ci = B.b2sr_to_csr(m)
        rp, ci = to_np(rp), to_np(ci)
        for g, b0 in zip(gs, bases[:-1]):
            want = oracle.canonicalize(g)
            grp = rp[b0:b0 + g.n + 1] - rp[b0]
            np.testing.assert_array_equal(grp, want.rowptr)
            np.testing.assert_array_equal(ci[rp[b0]:rp[b0 + g.n]] - b0, want.colind)
            # padding rows are empty
            assert rp[b0 + g.n] == rp[b0 + -(-g.n // 32) * 32]


@pytest.mark.parametrize("k", KS)
def test_arena_bfs_one_source_per_graph(B, k):
    gs = uneven_graphs()
    rng = np.random.default_rng(5 + k)
    m, bases, _ = arena(B, gs, k)
    with m:
        srcs, owners = [], []
        for gi, (g, b0) in enumerate(zip(gs, bases[:-1])):
            if g.n > 0:
                srcs.append(b0 + int(rng.integers(g.n)))
                owners.append(gi)
        levels = to_np(B.b2sr_bfs_sources(m, srcs))
    for s, gi in zip(srcs, owners):
        g, b0 = gs[gi], bases[gi]
        np.testing.assert_array_equal(levels[b0:b0 + g.n], oracle.bfs(g, s - b0), err_msg=f"graph {gi}")
    for g, b0, b1 in zip(gs, bases[:-1], bases[1:]):
        assert (levels[b0 + g.n:b1] == -1).all()


@pytest.mark.parametrize("k", [8, 32])
def test_arena_multi_source_bfs(B, k):
    """bfs_multi on the arena: lane s explores only its own graph."""
    gs = [g for g in uneven_graphs() if g.n > 0][:40]
    m, bases, _ = arena(B, gs, k)
    rng = np.random.default_rng(11)
    with m:
        srcs = [bases[i] + int(rng.integers(g.n)) for i, g in enumerate(gs)]
        lv = to_np(B.b2sr_bfs_multi(m, srcs))
    for s, (g, b0, b1) in enumerate(zip(gs, bases[:-1], bases[1:])):
        row = lv[s]
        np.testing.assert_array_equal(row[b0:b0 + g.n], oracle.bfs(g, srcs[s] - b0))
        assert (row[:b0] == -1).all() and (row[b0 + g.n:] == -1).all()


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("nsrc", [1, 2, 7, 64])
def test_bfs_sources_is_min_over_sources(B, k, nsrc):
    g = graphs.rmat(12, 16, seed=1)
    srcs = graphs.sources(g, nsrc, seed=nsrc)
    srcs = np.concatenate([srcs, srcs[:1]])   # a repeated source
    want = None
    for s in srcs:
        lv = oracle.bfs(g, int(s)).astype(np.int64)
        lv[lv < 0] = 1 << 40
        want = lv if want is None else np.minimum(want, lv)
    want[want == 1 << 40] = -1
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        got = to_np(B.b2sr_bfs_sources(m, srcs.tolist()))
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("n", [3, 5, 6, 7, 2049])
def test_captured_loop_depths(B, n):
    """Path depths around the four-round replay boundary and a deep path."""
    g = graphs.path(n)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        np.testing.assert_array_equal(to_np(B.b2sr_bfs(m, 0)), np.arange(n))
        d = to_np(B.b2sr_sssp(m, 0))
        np.testing.assert_array_equal(d, np.arange(n, dtype=np.float32))


def test_bfs_sources_not_converged(B):
    g = graphs.path(50)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        with pytest.raises(B.B2SRError):
            B.b2sr_bfs_sources(m, [0], max_iters=10)
        # exactly enough levels succeeds
        np.testing.assert_array_equal(to_np(B.b2sr_bfs_sources(m, [0], max_iters=49)), np.arange(50))


def test_bfs_sources_rejects_bad_sources(B):
    g = graphs.path(10)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        with pytest.raises(B.B2SRError):
            B.b2sr_bfs_sources(m, [3, 10])
        with pytest.raises(B.B2SRError):
            B.b2sr_bfs_sources(m, [])


def test_launches_counted_per_replay(B):
    g = graphs.path(40)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        B.b2sr_bfs(m, 0)
        torch.cuda.synchronize()
        l0 = B.b2sr_launch_count()
        B.b2sr_bfs(m, 0)
        short = B.b2sr_launch_count() - l0
    g2 = graphs.path(400)
    rp2, ci2 = csr_dev(g2)
    with B.b2sr_from_csr(g2.n, rp2, ci2, 8) as m2:
        l0 = B.b2sr_launch_count()
        B.b2sr_bfs(m2, 0)
        long = B.b2sr_launch_count() - l0
    assert long > 5 * short > 0


def test_arena_rejects_a_malformed_graph(B):
    """Each graph's own CSR is validated before it is shifted into the arena,
    so a column outside [0, n_g) is refused instead of becoming an edge into
    the next graph: a column equal to n_1 in graph 1, a negative column in
    graph 2, a last row pointer that disagrees with nnz, and a column in a
    graph with no vertices.  The error names the graph."""
    good = [graphs.path(40), graphs.cycle(33), graphs.star(50)]

    def build(mutate):
        csrs = []
        for i, g in enumerate(good):
            rp, ci = g.rowptr.copy(), g.colind.copy()
            rp, ci, n = mutate(i, rp, ci, g.n)
            csrs.append((n, torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda()))
        return B.b2sr_from_csr_batch(csrs, 8)

    def col_eq_n(i, rp, ci, n):
        if i == 1:
            ci[0] = n
        return rp, ci, n

    def negative(i, rp, ci, n):
        if i == 2:
            ci[-1] = -1
        return rp, ci, n

    def short_rowptr(i, rp, ci, n):
        if i == 1:
            rp[-1] -= 1
        return rp, ci, n

    def empty_with_col(i, rp, ci, n):
        if i == 0:
            return np.zeros(1, np.int32), np.array([0], np.int32), 0
        return rp, ci, n

    for mutate, gi in ((col_eq_n, 1), (negative, 2), (short_rowptr, 1), (empty_with_col, 0)):
        with pytest.raises(B.B2SRError, match=f"graph {gi}"):
            build(mutate)
    m, bases = build(lambda i, rp, ci, n: (rp, ci, n))   # the unmodified graphs still pack
    m.close()
