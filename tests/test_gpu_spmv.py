"""GPU parity: every SpMV scheme (Table 2) over every semiring (Table 4), all
tile sizes, with and without masks, element by element against the oracle.
Bit-exact for Boolean, integer and min outputs; fp32 plus-times within 1e-5
relative error of the fp64 oracle.  The tolerance follows from the kernel's
arithmetic: with non-negative inputs, a fixed-order fp32 sum of m terms has
relative error at most about m * 2^-24; each lane adds at most P*k = 64 set
bits in sequence, the warp joins 32 lanes in a 5-level tree, and partials of
rows that cross chunks are joined by a compensated (TwoSum) fp32 sum, which
adds at most 2 roundings, so m <= 71 and the bound is 71 * 2^-24 = 4.2e-6 <
1e-5."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import GRAPH_IDS, csr_dev, small_graphs, to_dev, to_np

pytestmark = pytest.mark.gpu

KS = [4, 8, 16, 32]
RTOL_F32 = 1e-5


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


@pytest.fixture(scope="module")
def mats(B):
    cache = {}

    def get(gi, k):
        if (gi, k) not in cache:
            g = small_graphs()[gi]
            rp, ci = csr_dev(g)
            cache[(gi, k)] = (g, B.b2sr_from_csr(g.n, rp, ci, k))
        return cache[(gi, k)]
    yield get
    for _, m in cache.values():
        m.close()


def canon(g):
    return oracle.canonicalize(g)


MASKS = [None, False, True]
SCHEDS = [1, 2]   # b2sr_schedule STAGED, DIRECT (the same at k = 32)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("masked", MASKS, ids=["nomask", "mask", "complement"])
def test_bool_and_count(B, mats, k, gi, masked):
    g, m = mats(gi, k)
    words = B.bitset_words(g.n)
    xb = graphs.random_bits(g.n, 0.05, seed=gi + 17)
    mask = None if masked is None else graphs.random_bits(g.n, 0.5, seed=gi + 29)
    y = torch.full((max(words, 1),), -1, dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, to_dev(xb), B.VEC_BITS, y,
                None if mask is None else to_dev(mask), bool(masked))
    np.testing.assert_array_equal(to_np(y, np.uint32)[:words], oracle.spmv_bool(canon(g), xb, mask, bool(masked)))
    yc = torch.full((max(g.n, 1),), -7, dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_BITS, to_dev(xb), B.VEC_I32, yc,
                None if mask is None else to_dev(mask), bool(masked))
    np.testing.assert_array_equal(to_np(yc)[: g.n], oracle.spmv_count(canon(g), xb, mask, bool(masked)))


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
def test_plus_times(B, mats, k, gi, sched):
    g, m = mats(gi, k)
    B.b2sr_set_schedule(m, sched)
    x = np.random.default_rng(gi).random(g.n).astype(np.float32)
    y = torch.full((max(g.n, 1),), float("nan"), dtype=torch.float32, device="cuda")
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, y)
    ref = oracle.spmv_plus(canon(g), x.astype(np.float64))
    got = to_np(y)[: g.n].astype(np.float64)
    np.testing.assert_allclose(got, ref, rtol=RTOL_F32, atol=0)
    # fixed reduction order: bitwise reproducible
    y2 = torch.empty_like(y)
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, y2)
    assert torch.equal(y, y2)
    mask = graphs.random_bits(g.n, 0.5, seed=gi)
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, y, to_dev(mask), True)
    refm = oracle.spmv_plus(canon(g), x.astype(np.float64), mask, True)
    np.testing.assert_allclose(to_np(y)[: g.n].astype(np.float64), refm, rtol=RTOL_F32, atol=0)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
def test_min_plus_unit_and_labels(B, mats, k, gi, sched):
    g, m = mats(gi, k)
    B.b2sr_set_schedule(m, sched)
    rng = np.random.default_rng(gi + 3)
    x = (rng.integers(0, 1000, g.n) / 4).astype(np.float32)   # exact sums
    x[rng.random(g.n) < 0.3] = np.inf
    y = torch.empty((max(g.n, 1),), dtype=torch.float32, device="cuda")
    B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_F32, to_dev(x), B.VEC_F32, y)
    np.testing.assert_array_equal(to_np(y)[: g.n], oracle.spmv_minplus(canon(g), x.astype(np.float64)).astype(np.float32))
    mask = graphs.random_bits(g.n, 0.5, seed=gi)
    B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_F32, to_dev(x), B.VEC_F32, y, to_dev(mask), False)
    np.testing.assert_array_equal(to_np(y)[: g.n],
                                  oracle.spmv_minplus(canon(g), x.astype(np.float64), None, mask, False).astype(np.float32))
    lab = rng.permutation(g.n).astype(np.int32)
    yi = torch.empty((max(g.n, 1),), dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_I32, to_dev(lab), B.VEC_I32, yi)
    np.testing.assert_array_equal(to_np(yi)[: g.n], oracle.spmv_min_i32(canon(g), lab))


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", [0, 2, 3, 4, 5], ids=["rmat12", "star20k", "grid37x41", "gaps", "directed300"])
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
def test_min_plus_weighted(B, mats, k, gi, sched):
    g, m = mats(gi, k)
    B.b2sr_set_schedule(m, sched)
    gc = canon(g)
    rng = np.random.default_rng(gi + 11)
    w_grid = (1 + rng.integers(0, 99 * 16, gc.colind.size) / 16).astype(np.float32)   # exact sums
    w_cont = rng.uniform(1.0, 100.0, gc.colind.size).astype(np.float32)
    x = (rng.integers(0, 4000, g.n) / 8).astype(np.float32)
    x[rng.random(g.n) < 0.2] = np.inf
    rp, ci = to_dev(gc.rowptr), to_dev(gc.colind)
    for w, exact in ((w_grid, True), (w_cont, False)):
        wb = B.b2sr_weights_from_csr(m, rp, ci, to_dev(w))
        y = torch.empty((max(g.n, 1),), dtype=torch.float32, device="cuda")
        B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_F32, to_dev(x), B.VEC_F32, y, weights=wb)
        ref = oracle.spmv_minplus(gc, x.astype(np.float64), w)
        got = to_np(y)[: g.n]
        if exact:
            np.testing.assert_array_equal(got, ref.astype(np.float32))
        else:
            fin = np.isfinite(ref)
            assert (np.isfinite(got) == fin).all()
            np.testing.assert_allclose(got[fin].astype(np.float64), ref[fin], rtol=RTOL_F32)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("masked", MASKS, ids=["nomask", "mask", "complement"])
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
def test_or64(B, mats, k, gi, masked, sched):
    g, m = mats(gi, k)
    B.b2sr_set_schedule(m, sched)
    rng = np.random.default_rng(gi + 5)
    X = rng.integers(0, 2**63, g.n, dtype=np.int64).astype(np.uint64)
    X[rng.random(g.n) < 0.7] = 0
    M = None if masked is None else rng.integers(0, 2**63, g.n, dtype=np.int64).astype(np.uint64)
    Y = torch.empty((max(g.n, 1),), dtype=torch.int64, device="cuda")
    B.b2sr_spmm_bits64(m, to_dev(X), Y, None if M is None else to_dev(M), bool(masked))
    np.testing.assert_array_equal(to_np(Y, np.uint64)[: g.n], oracle.spmm_or64(canon(g), X, M, bool(masked)))


def test_bad_combinations(B, mats):
    g, m = mats(0, 8)
    x = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    y = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    with pytest.raises(B.B2SRError):
        B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_F32, x, B.VEC_F32, y)
    with pytest.raises(B.B2SRError):
        B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, x, B.VEC_F32, x)
    with pytest.raises(B.B2SRError):
        B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, x, B.VEC_F32, y, weights=x)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
def test_plus_block_of_four(B, mats, k, gi, sched):
    """b2sr_spmm_f32x4: every column bitwise equal to the single-column
    plus-times SpMV, and within the fp32 tolerance of the oracle."""
    g, m = mats(gi, k)
    B.b2sr_set_schedule(m, sched)
    X = np.random.default_rng(gi + 40).random((g.n, 4)).astype(np.float32)
    X[:, 3] = 0.0                                   # an all-zero column
    Y = torch.full((max(g.n, 1), 4), float("nan"), dtype=torch.float32, device="cuda")
    B.b2sr_spmm_f32x4(m, to_dev(X if g.n else np.zeros((1, 4), np.float32)), Y)
    got = to_np(Y)[: g.n]
    for b in range(4):
        y1 = torch.empty(max(g.n, 1), dtype=torch.float32, device="cuda")
        B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(np.ascontiguousarray(X[:, b])), B.VEC_F32, y1)
        np.testing.assert_array_equal(got[:, b].view(np.uint32), to_np(y1)[: g.n].view(np.uint32))
        ref = oracle.spmv_plus(canon(g), X[:, b].astype(np.float64))
        np.testing.assert_allclose(got[:, b].astype(np.float64), ref, rtol=RTOL_F32, atol=0)
    mask = graphs.random_bits(g.n, 0.5, seed=gi + 41)
    B.b2sr_spmm_f32x4(m, to_dev(X if g.n else np.zeros((1, 4), np.float32)), Y, to_dev(mask), True)
    refm = oracle.spmv_plus(canon(g), X[:, 0].astype(np.float64), mask, True)
    np.testing.assert_allclose(to_np(Y)[: g.n, 0].astype(np.float64), refm, rtol=RTOL_F32, atol=0)


def test_plus_block_rejects_misaligned(B, mats):
    g, m = mats(0, 8)
    X = torch.zeros(4 * g.n + 1, dtype=torch.float32, device="cuda")
    Y = torch.zeros(4 * g.n, dtype=torch.float32, device="cuda")
    with pytest.raises(B.B2SRError):
        B.b2sr_spmm_f32x4(m, X[1:], Y)
