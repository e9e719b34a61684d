"""Oracle pins for short-bit-width weights held as bit-planes (Sec. VII:
W = sum_p 2^p A_p with binary A_p): the plane decomposition against the
pinned B2SR builder and against dense recombination; the weighted SpMVs
against dense numpy products and, for unit weights, against the pinned
unweighted SpMVs."""
import numpy as np
import pytest

import oracle
from paper_2201_08560_gb300 import graphs

GS = [graphs.rmat(9, 8, seed=3), graphs.random_directed(75, 0.1, seed=4), graphs.grid2d(9, 13),
      graphs.from_dense(np.zeros((10, 10)))]


def weights(g, bits, seed):
    return np.random.default_rng(seed).integers(0, 1 << bits, g.colind.size).astype(np.uint32)


def dense_w(g, w):
    W = np.zeros((g.n, g.n), dtype=np.int64)
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    W[rows, g.colind] = w
    return W


@pytest.mark.parametrize("k", [4, 8, 16, 32])
@pytest.mark.parametrize("gi", range(len(GS)))
def test_unit_and_power_weights_reproduce_the_pattern(k, gi):
    g = oracle.canonicalize(GS[gi])
    _, _, base = oracle.b2sr(g, k)
    one = np.ones(g.colind.size, np.uint32)
    np.testing.assert_array_equal(oracle.b2sr_planes(g, one, 1, k)[:, 0, :], base)
    P = oracle.b2sr_planes(g, one << 3, 5, k)
    for p in range(5):
        np.testing.assert_array_equal(P[:, p, :], base if p == 3 else np.zeros_like(base))


@pytest.mark.parametrize("k", [4, 8, 16, 32])
@pytest.mark.parametrize("gi", range(len(GS)))
@pytest.mark.parametrize("bits", [1, 3, 8, 16])
def test_planes_recombine_to_the_weights(k, gi, bits):
    g = oracle.canonicalize(GS[gi])
    w = weights(g, bits, gi + bits)
    trp, tci, _ = oracle.b2sr(g, k)
    P = oracle.b2sr_planes(g, w, bits, k)
    ntr = len(trp) - 1
    W = np.zeros((ntr * k, ntr * k), dtype=np.int64)
    for I in range(ntr):
        for t in range(trp[I], trp[I + 1]):
            J = tci[t]
            for p in range(bits):
                for r in range(k):
                    row = int(P[t, p, r])
                    for c in range(k):
                        if (row >> c) & 1:
                            W[I * k + r, J * k + c] += 1 << p
    np.testing.assert_array_equal(W[: g.n, : g.n], dense_w(g, w))
    assert not W[g.n:].any() and not W[:, g.n:].any()


def test_weight_too_wide_rejected():
    g = oracle.canonicalize(GS[0])
    w = weights(g, 4, 1)
    w[5] = 16
    with pytest.raises(ValueError):
        oracle.b2sr_planes(g, w, 4, 8)


@pytest.mark.parametrize("gi", range(len(GS)))
@pytest.mark.parametrize("masked", [None, False, True])
def test_weighted_spmvs_match_dense(gi, masked):
    g = oracle.canonicalize(GS[gi])
    w = weights(g, 16, gi)
    W = dense_w(g, w)
    xb = graphs.random_bits(g.n, 0.4, seed=gi)
    xv = graphs.unpack_bits(xb, g.n).astype(np.int64)
    mask = None if masked is None else graphs.random_bits(g.n, 0.5, seed=gi + 7)
    keep = np.ones(g.n, bool) if mask is None else graphs.unpack_bits(mask, g.n).astype(bool) ^ bool(masked)
    np.testing.assert_array_equal(oracle.spmv_wcount(g, w, xb, mask, bool(masked)), np.where(keep, W @ xv, 0))
    x = np.random.default_rng(gi).integers(0, 1000, g.n) / 4.0      # exact in fp64
    np.testing.assert_array_equal(oracle.spmv_wplus(g, w, x, mask, bool(masked)), np.where(keep, W @ x, 0.0))


@pytest.mark.parametrize("gi", range(len(GS)))
def test_unit_weights_reduce_to_the_unweighted_spmvs(gi):
    g = oracle.canonicalize(GS[gi])
    one = np.ones(g.colind.size, np.uint32)
    xb = graphs.random_bits(g.n, 0.3, seed=gi)
    np.testing.assert_array_equal(oracle.spmv_wcount(g, one, xb), oracle.spmv_count(g, xb))
    x = np.random.default_rng(gi).random(g.n)
    np.testing.assert_array_equal(oracle.spmv_wplus(g, one, x), oracle.spmv_plus(g, x))
