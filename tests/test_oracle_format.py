"""Pins for the oracle's B2SR construction (Sec. III-A/B, Table 1).

Each check is against something other than the oracle itself: the storage
sizes the paper prints for mycielskian12, a dense brute-force tiling, the
single-entry layout that the bit-order reading defines, and CSR round trips.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2201_08560_gb300 import graphs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_mycielskian12_storage_matches_paper():
    """Sec. III-C prints CSR 3.12 MB and B2SR-4/8/16/32 675.70/361.46/358.89/429.89 KB."""
    gold = json.load(open(os.path.join(GOLDEN, "mycielskian12_sizes.json")))
    g = graphs.mycielski(12)
    assert g.n == gold["n"]
    assert g.nnz == 2 * gold["undirected_edges"]
    csr_bytes = 4 * (g.n + 1) + 8 * g.nnz  # int32 rowptr + int32 colind + fp32 values
    assert round(csr_bytes / 2**20, 2) == gold["csr_mib"]
    for k in oracle.KS:
        trp, tci, tiles = oracle.b2sr(g, k)
        T = len(tci)
        got = oracle.b2sr_bytes(g.n, k, T)
        assert got == 4 * (len(trp)) + 4 * T + tiles.nbytes
        assert round(got / 1024, 2) == pytest.approx(gold["b2sr_kib"][str(k)], abs=0.005), k


def _dense_tile_counts(a: np.ndarray, k: int):
    n = a.shape[0]
    ntr = (n + k - 1) // k
    pad = np.zeros((ntr * k, ntr * k), dtype=bool)
    pad[:n, :n] = a != 0
    blocks = pad.reshape(ntr, k, ntr, k).any(axis=(1, 3))
    return blocks


@pytest.mark.parametrize("k", oracle.KS)
@pytest.mark.parametrize("n,density,seed", [(1, 1.0, 0), (7, 0.3, 1), (33, 0.1, 2), (64, 0.05, 3),
                                             (100, 0.02, 4), (37, 0.0, 5)])
def test_tiling_matches_dense_blocks(k, n, density, seed):
    """TileRowPtr/TileColInd = the non-empty k x k blocks of the dense matrix, in order."""
    g = graphs.random_directed(n, density, seed)
    a = graphs.to_dense(g)
    blocks = _dense_tile_counts(a, k)
    trp, tci, tiles = oracle.b2sr(g, k)
    assert trp[0] == 0 and len(trp) == blocks.shape[0] + 1
    np.testing.assert_array_equal(np.diff(trp), blocks.sum(axis=1))
    for I in range(blocks.shape[0]):
        np.testing.assert_array_equal(tci[trp[I]:trp[I + 1]], np.nonzero(blocks[I])[0])
    # every bit of every tile equals the dense entry it stands for; padding is zero
    ntr = blocks.shape[0]
    pad = np.zeros((ntr * k, ntr * k), dtype=np.int64)
    pad[:n, :n] = a
    for I in range(ntr):
        for t in range(trp[I], trp[I + 1]):
            J = tci[t]
            for r in range(k):
                word = int(tiles[t, r])
                for c in range(k):
                    assert ((word >> c) & 1) == pad[k * I + r, k * J + c]
                assert word >> k == 0


@pytest.mark.parametrize("k", oracle.KS)
def test_single_entry_layout(k):
    """Reading of the bit order: row word r of tile (I, J) holds row kI+r, bit c is column kJ+c."""
    n = 70
    for (i, j) in [(0, 0), (69, 3), (5, 66), (k, k - 1), (2 * k - 1, 0)]:
        if i >= n or j >= n:
            continue
        a = np.zeros((n, n), dtype=np.int64)
        a[i, j] = 1
        g = graphs.from_dense(a)
        trp, tci, tiles = oracle.b2sr(g, k)
        assert len(tci) == 1 and tci[0] == j // k
        assert trp[i // k] == 0 and trp[i // k + 1] == 1
        expect = np.zeros(k, dtype=np.int64)
        expect[i % k] = 1 << (j % k)
        np.testing.assert_array_equal(tiles[0].astype(np.int64), expect)


@pytest.mark.parametrize("k", oracle.KS)
def test_round_trip_with_duplicates_and_unsorted_rows(k):
    """CSR -> B2SR -> CSR returns the sorted, duplicate-free input pattern."""
    for seed, (n, dens) in enumerate([(50, 0.1), (129, 0.03), (31, 0.5), (1, 0.0)]):
        g = graphs.random_directed(n, dens, seed)
        gd = graphs.with_duplicates(g, seed + 10)
        trp, tci, tiles = oracle.b2sr(gd, k)
        back = oracle.b2sr_to_csr(n, k, trp, tci, tiles)
        np.testing.assert_array_equal(back.rowptr, g.rowptr)
        np.testing.assert_array_equal(back.colind, g.colind)
        canon = oracle.canonicalize(gd)
        np.testing.assert_array_equal(canon.rowptr, g.rowptr)
        np.testing.assert_array_equal(canon.colind, g.colind)


def test_invalid_inputs_rejected():
    g = graphs.path(5)
    with pytest.raises(ValueError):
        oracle.b2sr(g, 6)
    bad = graphs.CSR(5, g.rowptr.copy(), g.colind.copy())
    bad.colind[0] = 9
    with pytest.raises(ValueError):
        oracle.b2sr(bad, 8)
