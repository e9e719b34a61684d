"""GPU parity for bit-plane weights (Sec. VII: W = sum_p 2^p A_p): the
planes bit for bit against the oracle's decomposition, the weighted count
SpMV bit-exact (int64), the weighted plus-times SpMV within 1e-5 relative
error of the fp64 oracle (each term w_ij x_j is rounded once and the sums
are compensated, so the error stays near 2^-24 whatever the row length),
all tile sizes, with masks, on the small graphs and on a hub-heavy R-MAT."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import GRAPH_IDS, csr_dev, small_graphs, to_dev, to_np

pytestmark = pytest.mark.gpu

KS = [4, 8, 16, 32]
RTOL = 1e-5


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


def weights(g, bits, seed):
    return np.random.default_rng(seed).integers(0, 1 << bits, g.colind.size).astype(np.uint32)


def check(B, g, k, bits, seed, masked=None):
    g = oracle.canonicalize(g)
    w = weights(g, bits, seed)
    rp, ci = csr_dev(g)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        planes = B.b2sr_planes_from_csr(m, rp, ci, to_dev(w.view(np.int32)), bits)
        ref = oracle.b2sr_planes(g, w, bits, k)
        np.testing.assert_array_equal(to_np(planes)[: ref.nbytes], ref.reshape(-1).view(np.uint8))
        mask = None if masked is None else graphs.random_bits(g.n, 0.5, seed=seed + 1)
        dm = None if mask is None else to_dev(mask)
        xb = graphs.random_bits(g.n, 0.4, seed=seed + 2)
        y = torch.full((max(g.n, 1),), -5, dtype=torch.int64, device="cuda")
        B.b2sr_spmv_planes(m, planes, bits, B.VEC_BITS, to_dev(xb), B.VEC_I64, y, dm, bool(masked))
        np.testing.assert_array_equal(to_np(y)[: g.n], oracle.spmv_wcount(g, w, xb, mask, bool(masked)))
        x = np.random.default_rng(seed).random(g.n).astype(np.float32)
        yf = torch.full((max(g.n, 1),), float("nan"), dtype=torch.float32, device="cuda")
        B.b2sr_spmv_planes(m, planes, bits, B.VEC_F32, to_dev(x), B.VEC_F32, yf, dm, bool(masked))
        np.testing.assert_allclose(to_np(yf)[: g.n].astype(np.float64),
                                   oracle.spmv_wplus(g, w, x.astype(np.float64), mask, bool(masked)), rtol=RTOL, atol=0)
        yf2 = torch.empty_like(yf)
        B.b2sr_spmv_planes(m, planes, bits, B.VEC_F32, to_dev(x), B.VEC_F32, yf2, dm, bool(masked))
        assert torch.equal(yf, yf2)                                 # fixed order: reproducible


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("bits", [1, 5, 16])
def test_planes_small_graphs(B, k, gi, bits):
    check(B, small_graphs()[gi], k, bits, gi * 3 + bits)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("masked", [False, True], ids=["mask", "complement"])
def test_planes_masked(B, k, masked):
    check(B, small_graphs()[0], k, 8, 11, masked)


@pytest.mark.parametrize("k", [4, 8])
def test_planes_hub_rows(B, k):
    """R-MAT scale 16: tile-rows of more than 256 tiles go to the block kernel."""
    check(B, graphs.rmat(16, 16, seed=9), k, 8, 5)


def test_planes_errors(B):
    g = oracle.canonicalize(small_graphs()[3])
    rp, ci = csr_dev(g)
    w = weights(g, 4, 1)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        with pytest.raises(B.B2SRError, match="INVALID"):
            B.b2sr_planes_from_csr(m, rp, ci, to_dev(w.view(np.int32)), 3 if w.max() >= 8 else 0)
        with pytest.raises(B.B2SRError, match="INVALID"):
            B.b2sr_planes_from_csr(m, rp, ci, to_dev(w.view(np.int32)), 17)
        planes = B.b2sr_planes_from_csr(m, rp, ci, to_dev(w.view(np.int32)), 4)
        y = torch.empty(g.n, dtype=torch.int32, device="cuda")
        with pytest.raises(B.B2SRError, match="INVALID"):
            B.b2sr_spmv_planes(m, planes, 4, B.VEC_BITS, y, B.VEC_I32, y)
