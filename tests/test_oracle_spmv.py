"""Pins for the oracle's SpMV schemes (Table 2) over the Table 4 semirings.

Checked against dense brute force written with numpy matrix algebra on small
asymmetric matrices (so a transposed operand fails), with and without masks.
"""
import numpy as np
import pytest

import oracle
from paper_2201_08560_gb300 import graphs

CASES = [(1, 1.0, 0), (5, 0.4, 1), (33, 0.15, 2), (64, 0.08, 3), (97, 0.05, 4)]


def _mask_sel(n, mask_bits, complement):
    if mask_bits is None:
        return np.ones(n, dtype=bool)
    m = graphs.unpack_bits(mask_bits, n)
    return ~m if complement else m


@pytest.mark.parametrize("n,density,seed", CASES)
@pytest.mark.parametrize("masked", [None, False, True])
def test_bool_and_count(n, density, seed, masked):
    g = graphs.random_directed(n, density, seed)
    a = graphs.to_dense(g)
    xb = graphs.random_bits(n, 0.4, seed + 100)
    x = graphs.unpack_bits(xb, n).astype(np.int64)
    mask = None if masked is None else graphs.random_bits(n, 0.5, seed + 200)
    sel = _mask_sel(n, mask, bool(masked))
    expect_count = np.where(sel, a @ x, 0)
    expect_bool = (a @ x > 0) & sel
    yb = oracle.spmv_bool(g, xb, mask, bool(masked))
    np.testing.assert_array_equal(graphs.unpack_bits(yb, n), expect_bool)
    # bits beyond n are zero
    assert graphs.unpack_bits(yb, len(yb) * 32)[n:].sum() == 0
    np.testing.assert_array_equal(oracle.spmv_count(g, xb, mask, bool(masked)), expect_count)


@pytest.mark.parametrize("n,density,seed", CASES)
def test_plus_times(n, density, seed):
    g = graphs.random_directed(n, density, seed)
    a = graphs.to_dense(g).astype(np.float64)
    x = np.random.default_rng(seed).random(n)
    np.testing.assert_allclose(oracle.spmv_plus(g, x), a @ x, rtol=1e-15, atol=0)
    mask = graphs.random_bits(n, 0.5, seed + 1)
    sel = graphs.unpack_bits(mask, n)
    np.testing.assert_allclose(oracle.spmv_plus(g, x, mask, True), np.where(~sel, a @ x, 0.0),
                               rtol=1e-15, atol=0)


@pytest.mark.parametrize("n,density,seed", CASES)
@pytest.mark.parametrize("weighted", [False, True])
def test_min_plus(n, density, seed, weighted):
    g = graphs.random_directed(n, density, seed)
    a = graphs.to_dense(g)
    rng = np.random.default_rng(seed + 7)
    x = rng.random(n) * 10
    x[rng.random(n) < 0.2] = np.inf
    w = None
    wd = np.ones((n, n))
    if weighted:
        w = rng.uniform(0.0, 5.0, g.nnz).astype(np.float32)
        for i in range(n):
            for e in range(g.rowptr[i], g.rowptr[i + 1]):
                wd[i, g.colind[e]] = w[e]
    cand = np.where(a > 0, x[None, :] + wd, np.inf)
    expect = np.minimum(x, cand.min(axis=1) if n else x)
    np.testing.assert_array_equal(oracle.spmv_minplus(g, x, w), expect)
    mask = graphs.random_bits(n, 0.5, seed + 3)
    sel = graphs.unpack_bits(mask, n)
    np.testing.assert_array_equal(oracle.spmv_minplus(g, x, w, mask, False), np.where(sel, expect, np.inf))


@pytest.mark.parametrize("n,density,seed", CASES)
def test_min_labels(n, density, seed):
    g = graphs.random_directed(n, density, seed)
    a = graphs.to_dense(g)
    x = np.random.default_rng(seed).permutation(n).astype(np.int32)
    cand = np.where(a > 0, x[None, :], np.iinfo(np.int32).max)
    expect = np.minimum(x, cand.min(axis=1))
    np.testing.assert_array_equal(oracle.spmv_min_i32(g, x), expect)


@pytest.mark.parametrize("n,density,seed", CASES)
@pytest.mark.parametrize("mode", [None, False, True])
def test_or64(n, density, seed, mode):
    g = graphs.random_directed(n, density, seed)
    a = graphs.to_dense(g)
    rng = np.random.default_rng(seed + 11)
    X = rng.integers(0, 2**63, size=n, dtype=np.int64).astype(np.uint64) * np.uint64(2) + np.uint64(1)
    M = None if mode is None else rng.integers(0, 2**63, size=n, dtype=np.int64).astype(np.uint64)
    expect = np.zeros(n, dtype=np.uint64)
    for i in range(n):
        for j in range(n):
            if a[i, j]:
                expect[i] |= X[j]
    if M is not None:
        expect = expect & (~M if mode else M)
    np.testing.assert_array_equal(oracle.spmm_or64(g, X, M, bool(mode)), expect)


def test_row_loops_do_not_depend_on_thread_count():
    """The oracle's row loops run on any number of host threads (the CPU
    baseline is timed on one and on all); every row is still computed by one
    thread in CSR order, so each result is identical, bit for bit."""
    from paper_2201_08560_gb300 import graphs
    g = graphs.rmat(13, 16, seed=4)
    xb = graphs.random_bits(g.n, 0.1, seed=1)
    xf = np.random.default_rng(2).random(g.n)
    mask = graphs.random_bits(g.n, 0.5, seed=3)
    prev = oracle.set_threads(0)
    try:
        out = []
        for t in (1, max(2, prev)):
            oracle.set_threads(t)
            out.append([oracle.spmv_bool(g, xb, mask, True), oracle.spmv_count(g, xb), oracle.spmv_plus(g, xf),
                        oracle.spmv_minplus(g, xf), oracle.spmv_max(g, xf), oracle.pagerank(g, 0.85, 5)])
        for a, b in zip(*out):
            np.testing.assert_array_equal(a, b)
    finally:
        oracle.set_threads(prev)
