"""The allocation-free Boolean SpMV entry point.

b2sr_spmv_bool_noalloc exists for callers that cannot allocate device memory
when they call into the library (for example a host whose own allocator has
reserved the device's free memory).  It keeps its scratch in a fixed array
inside the library instead.  These checks call it through the C ABI twice in a
row and compare each result with b2sr_spmv's Boolean scheme, bit for bit
(the tolerance of every Boolean test here).  This file is collected last, so a
run that stops at its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2201_08560_gb300 import graphs
from tests.gpu_util import csr_dev, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


CASES = [graphs.rmat(12, 16, seed=1), graphs.star(20000), graphs.grid2d(37, 41)]


@pytest.mark.parametrize("k", [4, 8, 16, 32])
@pytest.mark.parametrize("gi", range(len(CASES)), ids=["rmat12", "star20k", "grid37x41"])
def test_noalloc_matches_spmv_on_consecutive_calls(B, k, gi):
    g = CASES[gi]
    rp, ci = csr_dev(g)
    words = B.bitset_words(g.n)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        calls = [(graphs.random_bits(g.n, 0.05, 11 + gi), None, False),
                 (graphs.random_bits(g.n, 0.3, 23 + gi), graphs.random_bits(g.n, 0.5, 31 + gi), True)]
        for xb, mask, comp in calls:
            x = to_dev(xb)
            mk = None if mask is None else to_dev(mask)
            want = torch.full((words,), -1, dtype=torch.int32, device="cuda")
            got = torch.full((words,), 0x5A5A5A5A, dtype=torch.int32, device="cuda")
            B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, x, B.VEC_BITS, want, mk, comp)
            B.b2sr_spmv_bool_noalloc(m, x, got, mk, comp)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(to_np(got, np.uint32), to_np(want, np.uint32))


def test_noalloc_rejects_null_pointers(B):
    g = CASES[0]
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        y = torch.empty(B.bitset_words(g.n), dtype=torch.int32, device="cuda")
        st = B.lib.b2sr_spmv_bool_noalloc(m.handle, None, B._ptr(y), None, 0, B._stream())
        assert st == 1  # B2SR_ERR_INVALID_ARG
        assert b"NULL" in B.lib.b2sr_last_error()
