"""The allocation-free Boolean SpMV entry point.

b2sr_spmv_bool_noalloc exists for callers that cannot allocate device memory
when they call into the library (for example a host whose own allocator has
reserved the device's free memory, or a service that must not allocate once
it runs).  It keeps its scratch in a fixed array inside the library instead.
These checks call it through the C ABI twice in a row, compare each result
with the CPU oracle and with b2sr_spmv's Boolean scheme, bit for bit (the
tolerance of every Boolean test here), run it on a matrix exactly at the
array's limit, and check that a matrix one tile past the limit is refused
before anything runs.  This file is collected last, so a run that stops at
its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import csr_dev, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


CASES = [graphs.rmat(12, 16, seed=1), graphs.star(20000), graphs.grid2d(37, 41)]


def _check_twice(B, g, m, seed):
    words = B.bitset_words(g.n)
    calls = [(graphs.random_bits(g.n, 0.05, 11 + seed), None, False),
             (graphs.random_bits(g.n, 0.3, 23 + seed), graphs.random_bits(g.n, 0.5, 31 + seed), True)]
    for xb, mask, comp in calls:
        x = to_dev(xb)
        mk = None if mask is None else to_dev(mask)
        want = torch.full((words,), -1, dtype=torch.int32, device="cuda")
        got = torch.full((words,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
        B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, x, B.VEC_BITS, want, mk, comp)
        B.b2sr_spmv_bool_noalloc(m, x, got, mk, comp)
        torch.cuda.synchronize()
        got_np = to_np(got, np.uint32)
        np.testing.assert_array_equal(got_np, oracle.spmv_bool(g, xb, mask, comp))
        np.testing.assert_array_equal(got_np, to_np(want, np.uint32))


@pytest.mark.parametrize("k", [4, 8, 16, 32])
@pytest.mark.parametrize("gi", range(len(CASES)), ids=["rmat12", "star20k", "grid37x41"])
def test_noalloc_matches_oracle_on_consecutive_calls(B, k, gi):
    g = CASES[gi]
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        _check_twice(B, g, m, gi)


def _limit_graph(extra_tile: bool):
    """A graph whose B2SR at tile_dim 32 has exactly 524,288 chunks of 64
    tiles (the fixed array's limit at k = 32): 2^25 vertices, 2^20 tile-rows
    of 32 tiles, each tile holding one bit of its tile-row's first row; with
    extra_tile, one more tile in tile-row 0 (one chunk too many)."""
    n = 1 << 25
    ntr = n // 32
    I = np.arange(ntr, dtype=np.int64)
    j = np.arange(32, dtype=np.int64)
    tcol = np.sort((I[:, None] * 37 + j[None, :] * 32771) % ntr, axis=1)   # 32 distinct tile-columns a row
    counts = np.zeros(n, dtype=np.int64)
    counts[I * 32] = 32
    parts = [tcol[0] * 32]
    if extra_tile:                       # row 1 (tile-row 0): one entry in a tile-column row 0 lacks
        spare = int(np.setdiff1d(np.arange(64), tcol[0])[0])
        counts[1] = 1
        parts.append(np.array([spare * 32 + 5]))
    parts.append(tcol[1:].reshape(-1) * 32)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return graphs.CSR(n, rowptr.astype(np.int32), np.concatenate(parts).astype(np.int32))


def test_noalloc_at_and_past_the_scratch_limit(B):
    g = _limit_graph(False)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 32) as m:
        assert m.n_tiles == 524288 * 64
        _check_twice(B, g, m, 100)
    del rp, ci
    g = _limit_graph(True)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 32) as m:
        assert m.n_tiles == 524288 * 64 + 1
        words = B.bitset_words(g.n)
        x = torch.zeros(words, dtype=torch.int32, device="cuda")
        y = torch.full((words,), 7, dtype=torch.int32, device="cuda")
        st = B.lib.b2sr_spmv_bool_noalloc(m.handle, B._ptr(x), B._ptr(y), None, 0, B._stream())
        assert st == 1  # B2SR_ERR_INVALID_ARG
        msg = B.lib.b2sr_last_error().decode()
        assert "524289 chunks" in msg and "4194304" in msg
        torch.cuda.synchronize()
        assert (y == 7).all()  # refused before anything ran


def test_noalloc_rejects_null_pointers(B):
    g = CASES[0]
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        y = torch.empty(B.bitset_words(g.n), dtype=torch.int32, device="cuda")
        st = B.lib.b2sr_spmv_bool_noalloc(m.handle, None, B._ptr(y), None, 0, B._stream())
        assert st == 1  # B2SR_ERR_INVALID_ARG
        assert b"NULL" in B.lib.b2sr_last_error()
