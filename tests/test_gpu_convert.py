"""GPU parity: CSR -> B2SR conversion, export, B2SR -> CSR, lower triangle
and the weight side array, element by element against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import GRAPH_IDS, csr_dev, dev, small_graphs, to_dev, to_np

pytestmark = pytest.mark.gpu

KS = [4, 8, 16, 32]


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


def _oracle_arrays(g, k):
    trp, tci, tiles = oracle.b2sr(g, k)
    return trp, tci, tiles.reshape(-1).view(np.uint8)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
def test_from_csr_matches_oracle(B, k, gi):
    g = small_graphs()[gi]
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        trp, tci, tiles = _oracle_arrays(g, k)
        assert m.n_tiles == len(tci)
        assert m.nnz == g.nnz
        assert m.bytes == oracle.b2sr_bytes(g.n, k, len(tci))
        grp, gci, gt = B.b2sr_export(m)
        np.testing.assert_array_equal(to_np(grp), trp)
        np.testing.assert_array_equal(to_np(gci), tci)
        np.testing.assert_array_equal(to_np(gt), tiles)
        r2, c2 = B.b2sr_to_csr(m)
        canon = oracle.canonicalize(g)
        np.testing.assert_array_equal(to_np(r2), canon.rowptr)
        np.testing.assert_array_equal(to_np(c2), canon.colind)


@pytest.mark.parametrize("k", KS)
def test_duplicates_and_unsorted_rows_are_ored(B, k):
    g = graphs.random_directed(203, 0.07, seed=5)
    gd = graphs.with_duplicates(g, seed=6)
    rp, ci = csr_dev(gd)
    with B.b2sr_from_csr(gd.n, rp, ci, k) as m:
        trp, tci, tiles = _oracle_arrays(g, k)
        grp, gci, gt = B.b2sr_export(m)
        np.testing.assert_array_equal(to_np(gci), tci)
        np.testing.assert_array_equal(to_np(gt), tiles)
        assert m.nnz == g.nnz


def _sort_rows(g):
    """The same CSR with every row in column order (repeats kept)."""
    ci = g.colind.copy()
    for i in range(g.n):
        ci[g.rowptr[i]:g.rowptr[i + 1]].sort()
    return graphs.CSR(g.n, g.rowptr.copy(), ci, None, g.name + "-sorted")


@pytest.mark.parametrize("k", KS)
def test_sorted_rows_with_repeats_and_hubs(B, k):
    """Column-ordered rows take the ranking conversion: repeated columns, a
    hub row far longer than its tile-row's other rows, and n not a multiple
    of k must still give the oracle's arrays."""
    g = graphs.disjoint_union(graphs.star(2503), graphs.random_directed(203, 0.07, seed=5),
                              graphs.rmat(9, 8, seed=3))
    gs = _sort_rows(graphs.with_duplicates(g, seed=7))
    assert all(np.all(np.diff(gs.colind[gs.rowptr[i]:gs.rowptr[i + 1]]) >= 0) for i in range(gs.n))
    assert gs.nnz > g.nnz and gs.n % 4 != 0
    rp, ci = csr_dev(gs)
    with B.b2sr_from_csr(gs.n, rp, ci, k) as m:
        trp, tci, tiles = _oracle_arrays(g, k)
        grp, gci, gt = B.b2sr_export(m)
        np.testing.assert_array_equal(to_np(grp), trp)
        np.testing.assert_array_equal(to_np(gci), tci)
        np.testing.assert_array_equal(to_np(gt), tiles)
        assert m.nnz == g.nnz


@pytest.mark.parametrize("k", KS)
def test_one_unsorted_row_gives_the_same_arrays(B, k):
    """One row out of column order sends the whole matrix down the sorting
    conversion; its arrays equal the sorted input's."""
    g = graphs.rmat(10, 8, seed=11)
    ci = g.colind.copy()
    i = int(np.argmax(np.diff(g.rowptr)))
    ci[g.rowptr[i]:g.rowptr[i + 1]] = ci[g.rowptr[i]:g.rowptr[i + 1]][::-1]
    gu = graphs.CSR(g.n, g.rowptr.copy(), ci, None, "rmat10-one-reversed")
    trp, tci, tiles = _oracle_arrays(g, k)
    for h in (g, gu):
        rp, cd = csr_dev(h)
        with B.b2sr_from_csr(h.n, rp, cd, k) as m:
            grp, gci, gt = B.b2sr_export(m)
            np.testing.assert_array_equal(to_np(grp), trp)
            np.testing.assert_array_equal(to_np(gci), tci)
            np.testing.assert_array_equal(to_np(gt), tiles)


@pytest.mark.parametrize("k", [4, 8])
def test_column_array_off_a_16_byte_boundary(B, k):
    """colind that starts 4 bytes past an aligned address (a view into a
    larger buffer): the validation's vector loads must not be used on it."""
    g = graphs.rmat(9, 8, seed=21)
    rp, ci = csr_dev(g)
    buf = torch.zeros(ci.numel() + 1, dtype=torch.int32, device=ci.device)
    buf[1:] = ci
    view = buf[1:]
    assert view.data_ptr() % 16 != 0
    trp, tci, tiles = _oracle_arrays(g, k)
    with B.b2sr_from_csr(g.n, rp, view, k) as m:
        grp, gci, gt = B.b2sr_export(m)
        np.testing.assert_array_equal(to_np(gci), tci)
        np.testing.assert_array_equal(to_np(gt), tiles)


def test_mycielskian12_sizes_from_gpu(B):
    """The paper's Sec. III-C storage sizes, produced by the GPU conversion."""
    g = graphs.mycielski(12)
    rp, ci = csr_dev(g)
    expect_kib = {4: 675.70, 8: 361.46, 16: 358.89, 32: 429.89}
    for k in KS:
        with B.b2sr_from_csr(g.n, rp, ci, k) as m:
            assert round(m.bytes / 1024, 2) == pytest.approx(expect_kib[k], abs=0.005)


def test_invalid_csr_rejected(B):
    g = graphs.path(10)
    rp, ci = csr_dev(g)
    bad = ci.clone()
    bad[3] = 99
    with pytest.raises(B.B2SRError) as e:
        B.b2sr_from_csr(g.n, rp, bad, 8)
    assert e.value.status == 1
    with pytest.raises(B.B2SRError) as e:
        B.b2sr_from_csr(g.n, rp, ci, 12)
    assert e.value.status == 2
    dec = rp.clone()
    dec[5] = 0
    with pytest.raises(B.B2SRError):
        B.b2sr_from_csr(g.n, dec, ci, 8)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", [0, 2, 4, 8], ids=["rmat12", "star20k", "gaps", "mycielski9"])
def test_lower_triangle(B, k, gi):
    g = small_graphs()[gi]
    a_lower = graphs.from_dense(np.tril(graphs.to_dense(g), -1)) if g.n <= 3000 else None
    if a_lower is None:
        rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
        keep = g.colind < rows
        a_lower = graphs.from_edges(g.n, rows[keep], g.colind[keep], symmetric=False, drop_self_loops=False)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m, B.b2sr_lower(m) as L:
        trp, tci, tiles = _oracle_arrays(a_lower, k)
        grp, gci, gt = B.b2sr_export(L)
        np.testing.assert_array_equal(to_np(grp), trp)
        np.testing.assert_array_equal(to_np(gci), tci)
        np.testing.assert_array_equal(to_np(gt), tiles)


@pytest.mark.parametrize("k", KS)
def test_weights_set_bit_order(B, k):
    g = graphs.grid2d(23, 29)
    w = graphs.symmetric_weights(g, seed=3)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        wb = to_np(B.b2sr_weights_from_csr(m, rp, ci, to_dev(w)))
        # expected: walk the oracle's tiles in (tile, row word, bit) order
        trp, tci, tiles = oracle.b2sr(g, k)
        lookup = {}
        for i in range(g.n):
            for e in range(g.rowptr[i], g.rowptr[i + 1]):
                lookup[(i, int(g.colind[e]))] = w[e]
        expect = []
        for I in range(len(trp) - 1):
            for t in range(trp[I], trp[I + 1]):
                for r in range(k):
                    word = int(tiles[t, r])
                    for c in range(k):
                        if (word >> c) & 1:
                            expect.append(lookup[(k * I + r, k * int(tci[t]) + c)])
        np.testing.assert_array_equal(wb, np.asarray(expect, dtype=np.float32))
