"""GPU parity for the max-times semiring (Table 4) and the two operations
Table 4 lists it for: the maximal independent set and graph colouring,
element by element against the oracle, bit-exact (max is exact; sets and
colours are integers).  Also: every bitset-masked SpMV with masks that leave
whole chunks of output rows excluded (the kernels skip those chunks' tiles)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import GRAPH_IDS, csr_dev, small_graphs, to_dev, to_np

pytestmark = pytest.mark.gpu

KS = [4, 8, 16, 32]
SCHEDS = [1, 2]   # STAGED, DIRECT


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


def symmetric(g):
    """The undirected graph of g (A | A^T), self-loops kept."""
    rows = np.repeat(np.arange(g.n), np.diff(g.rowptr))
    return graphs.from_edges(g.n, rows, g.colind, symmetric=True, drop_self_loops=False, name=g.name)


@pytest.fixture(scope="module")
def mats(B):
    cache = {}

    def get(gi, k, sym=False):
        key = (gi, k, sym)
        if key not in cache:
            g = small_graphs()[gi]
            if sym:
                g = symmetric(g)
            rp, ci = csr_dev(g)
            cache[key] = (oracle.canonicalize(g), B.b2sr_from_csr(g.n, rp, ci, k))
        return cache[key]
    yield get
    for _, m in cache.values():
        m.close()


def priorities(n, kind, seed):
    rng = np.random.default_rng(seed)
    if kind == "distinct":
        return rng.permutation(n).astype(np.float32) + 1.0
    if kind == "ties":                       # ties broken by the larger id
        return rng.integers(0, 4, n).astype(np.float32)
    if kind == "zeros":                      # +0 and -0 compare equal
        return rng.choice(np.array([0.0, -0.0, 1.5, -2.0], np.float32), n)
    p = rng.normal(size=n).astype(np.float32)  # with infinities
    p[rng.random(n) < 0.1] = np.inf
    p[rng.random(n) < 0.1] = -np.inf
    return p


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("masked", [None, False, True], ids=["nomask", "mask", "complement"])
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
def test_max_times(B, mats, k, gi, masked, sched):
    g, m = mats(gi, k)
    B.b2sr_set_schedule(m, sched)
    rng = np.random.default_rng(gi + 41)
    x = rng.normal(size=g.n).astype(np.float32)
    x[rng.random(g.n) < 0.1] = -np.inf
    x[rng.random(g.n) < 0.02] = np.inf
    mask = None if masked is None else graphs.random_bits(g.n, 0.5, seed=gi + 3)
    y = torch.full((max(g.n, 1),), float("nan"), dtype=torch.float32, device="cuda")
    B.b2sr_spmv(m, B.MAX_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, y,
                None if mask is None else to_dev(mask), bool(masked))
    ref = oracle.spmv_max(g, x.astype(np.float64), mask, bool(masked)).astype(np.float32)
    np.testing.assert_array_equal(to_np(y)[: g.n], ref)
    B.b2sr_set_schedule(m, 0)


def test_max_times_rejects_weights(B, mats):
    g, m = mats(0, 8)
    x = torch.zeros(g.n, dtype=torch.float32, device="cuda")
    w = torch.ones(m.nnz, dtype=torch.float32, device="cuda")
    with pytest.raises(B.B2SRError):
        B.b2sr_spmv(m, B.MAX_TIMES, B.VEC_F32, x, B.VEC_F32, torch.empty_like(x), weights=w)
    with pytest.raises(B.B2SRError):
        B.b2sr_spmv(m, B.MAX_TIMES, B.VEC_I32, x.int(), B.VEC_I32, torch.empty_like(x).int())


KINDS = ["distinct", "ties", "zeros", "infinite"]


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
def test_mis(B, mats, k, gi, kind, sched):
    g, m = mats(gi, k, sym=True)
    B.b2sr_set_schedule(m, sched)
    pr = priorities(g.n, kind, gi + 7)
    got = to_np(B.b2sr_mis(m, to_dev(pr)))
    np.testing.assert_array_equal(got, oracle.mis_greedy(g, pr.astype(np.float64)))
    B.b2sr_set_schedule(m, 0)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
def test_color_max_times(B, mats, k, gi, kind, sched):
    g, m = mats(gi, k, sym=True)
    B.b2sr_set_schedule(m, sched)
    pr = priorities(g.n, kind, gi + 13)
    got = to_np(B.b2sr_color(m, to_dev(pr), method=B.COLOR_MAX_TIMES))
    np.testing.assert_array_equal(got, oracle.color_levels(g, pr.astype(np.float64)))
    B.b2sr_set_schedule(m, 0)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("kind", KINDS)
def test_color_push(B, mats, k, gi, kind):
    g, m = mats(gi, k, sym=True)
    pr = priorities(g.n, kind, gi + 13)
    ref = oracle.color_levels(g, pr.astype(np.float64))
    np.testing.assert_array_equal(to_np(B.b2sr_color(m, to_dev(pr), method=B.COLOR_PUSH)), ref)
    np.testing.assert_array_equal(to_np(B.b2sr_color(m, to_dev(pr))), ref)          # AUTO


@pytest.mark.parametrize("k", [4, 8])
def test_mis_and_color_rmat16(B, k):
    g = graphs.rmat(16, 16, seed=5)
    rp, ci = csr_dev(g)
    pr = priorities(g.n, "distinct", 3)
    with B.b2sr_from_csr(g.n, rp, ci, k) as m:
        s = to_np(B.b2sr_mis(m, to_dev(pr)))
        c = to_np(B.b2sr_color(m, to_dev(pr), method=B.COLOR_PUSH))
        c2 = to_np(B.b2sr_color(m, to_dev(pr), method=B.COLOR_MAX_TIMES))
    np.testing.assert_array_equal(s, oracle.mis_greedy(g, pr.astype(np.float64)))
    ref = oracle.color_levels(g, pr.astype(np.float64))
    np.testing.assert_array_equal(c, ref)
    np.testing.assert_array_equal(c2, ref)


def test_mis_color_errors(B, mats):
    g, m = mats(3, 8, sym=True)                          # grid 37 x 41
    pr = priorities(g.n, "distinct", 1)
    bad = pr.copy()
    bad[100] = np.nan
    with pytest.raises(B.B2SRError, match="INVALID"):
        B.b2sr_mis(m, to_dev(bad))
    with pytest.raises(B.B2SRError, match="INVALID"):
        B.b2sr_color(m, to_dev(bad))
    with pytest.raises(B.B2SRError, match="INVALID"):
        B.b2sr_color(m, to_dev(bad), method=B.COLOR_MAX_TIMES)
    with pytest.raises(B.B2SRError, match="INVALID"):
        B.b2sr_color(m, to_dev(pr), method=7)
    with pytest.raises(ValueError):
        B.b2sr_mis(m, to_dev(pr.astype(np.float64)))
    path = graphs.path(300)                              # falling priorities: 300 colours
    rp, ci = csr_dev(path)
    with B.b2sr_from_csr(path.n, rp, ci, 8) as mp:
        fall = (1000.0 - np.arange(300)).astype(np.float32)
        for method in (B.COLOR_MAX_TIMES, B.COLOR_PUSH):
            with pytest.raises(B.B2SRError, match="NOT_CONVERGED"):
                B.b2sr_color(mp, to_dev(fall), method=method, max_iters=16)
            np.testing.assert_array_equal(to_np(B.b2sr_color(mp, to_dev(fall), method=method)), np.arange(300))
        np.testing.assert_array_equal(to_np(B.b2sr_mis(mp, to_dev(fall))), np.arange(300) % 2 == 0)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("gi", range(len(GRAPH_IDS)), ids=GRAPH_IDS)
@pytest.mark.parametrize("sched", SCHEDS, ids=["staged", "direct"])
@pytest.mark.parametrize("comp", [False, True], ids=["mask", "complement"])
def test_mostly_excluding_masks(B, mats, k, gi, sched, comp):
    """Masks that exclude nearly every row, so most chunks have no row to
    store: every bitset-masked semiring still matches the oracle."""
    g, m = mats(gi, k)
    B.b2sr_set_schedule(m, sched)
    dens = 0.995 if comp else 0.005
    mask = graphs.random_bits(g.n, dens, seed=gi + 101)
    dm = to_dev(mask)
    rng = np.random.default_rng(gi + 77)
    n1 = max(g.n, 1)
    xb = graphs.random_bits(g.n, 0.2, seed=gi + 5)
    y = torch.full((B.bitset_words(g.n) or 1,), -1, dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, to_dev(xb), B.VEC_BITS, y, dm, comp)
    np.testing.assert_array_equal(to_np(y, np.uint32)[: B.bitset_words(g.n)], oracle.spmv_bool(g, xb, mask, comp))
    yc = torch.full((n1,), -7, dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_BITS, to_dev(xb), B.VEC_I32, yc, dm, comp)
    np.testing.assert_array_equal(to_np(yc)[: g.n], oracle.spmv_count(g, xb, mask, comp))
    x = (rng.integers(0, 1000, g.n) / 4).astype(np.float32)        # exact sums
    yf = torch.full((n1,), float("nan"), dtype=torch.float32, device="cuda")
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, yf, dm, comp)
    np.testing.assert_array_equal(to_np(yf)[: g.n], oracle.spmv_plus(g, x.astype(np.float64), mask, comp).astype(np.float32))
    B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_F32, to_dev(x), B.VEC_F32, yf, dm, comp)
    np.testing.assert_array_equal(to_np(yf)[: g.n],
                                  oracle.spmv_minplus(g, x.astype(np.float64), None, mask, comp).astype(np.float32))
    B.b2sr_spmv(m, B.MAX_TIMES, B.VEC_F32, to_dev(x), B.VEC_F32, yf, dm, comp)
    np.testing.assert_array_equal(to_np(yf)[: g.n], oracle.spmv_max(g, x.astype(np.float64), mask, comp).astype(np.float32))
    lab = rng.permutation(g.n).astype(np.int32)
    B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_I32, to_dev(lab), B.VEC_I32, yc, dm, comp)
    np.testing.assert_array_equal(to_np(yc)[: g.n], oracle.spmv_min_i32(g, lab, mask, comp))
    B.b2sr_set_schedule(m, 0)
