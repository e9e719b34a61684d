"""GPU parity for tile size selection (Sec. III-C, Algorithm 1): the device
sampling estimate against the oracle's, and the autotuner's choice checked
for consistency (the returned handle is the candidate its own trials found
fastest, and it computes what the oracle computes)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import GRAPH_IDS, csr_dev, small_graphs, to_dev, to_np

pytestmark = pytest.mark.gpu

KS = [4, 8, 16, 32]


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


def samples(n, seed):
    rng = np.random.default_rng(seed)
    return [np.arange(n, dtype=np.int32),                              # every row once
            rng.integers(0, n, max(1, n // 10)).astype(np.int32),      # 10% with repeats
            rng.integers(0, n, 7).astype(np.int32)]


@pytest.mark.parametrize("gi", [i for i, name in enumerate(GRAPH_IDS) if name != "empty45"] , ids=[
    name for name in GRAPH_IDS if name != "empty45"])
def test_sample_profile_matches_oracle(B, gi):
    g = small_graphs()[gi]
    rp, ci = csr_dev(g)
    for smp in samples(g.n, gi):
        est, th = B.b2sr_sample_profile(g.n, rp, ci, smp)
        oest, oth = oracle.sample_profile(g, smp)
        # integer counts scaled identically: the tile estimate is bit-exact; the
        # ratio may differ in the last place where a host compiler fuses a multiply-add
        np.testing.assert_array_equal(np.array(th), oth)
        np.testing.assert_allclose(np.array(est), oest, rtol=1e-12, atol=0)


def test_sample_profile_full_sample_counts_tiles(B):
    g = graphs.rmat(12, 16, seed=1)          # n = 4096, divisible by every k
    rp, ci = csr_dev(g)
    _, th = B.b2sr_sample_profile(g.n, rp, ci, np.arange(g.n, dtype=np.int32))
    for q, k in enumerate(KS):
        with B.b2sr_from_csr(g.n, rp, ci, k) as m:
            assert th[q] == m.n_tiles


def test_sample_profile_unsorted_duplicated_rows(B):
    g = graphs.with_duplicates(graphs.rmat(10, 8, seed=3), seed=4)
    rp, ci = csr_dev(g)
    smp = np.random.default_rng(0).integers(0, g.n, 300).astype(np.int32)
    est, th = B.b2sr_sample_profile(g.n, rp, ci, smp)
    oest, oth = oracle.sample_profile(g, smp)
    np.testing.assert_array_equal(np.array(th), oth)


def test_sample_profile_rejects_bad_rows(B):
    g = graphs.path(10)
    rp, ci = csr_dev(g)
    with pytest.raises(B.B2SRError):
        B.b2sr_sample_profile(g.n, rp, ci, np.array([0, 10], np.int32))
    with pytest.raises(B.B2SRError):
        B.b2sr_sample_profile(g.n, rp, ci, np.array([-1], np.int32))


@pytest.mark.parametrize("scheme", ["bool", "plus", "minplus"])
@pytest.mark.parametrize("keep", [0.0, 1.5])
def test_autotune_choice_is_consistent(B, scheme, keep):
    g = graphs.rmat(13, 16, seed=5)
    rp, ci = csr_dev(g)
    sr, vk = {"bool": (B.BOOL_OR_AND, B.VEC_BITS), "plus": (B.PLUS_TIMES, B.VEC_F32),
              "minplus": (B.MIN_PLUS, B.VEC_F32)}[scheme]
    smp = np.random.default_rng(1).integers(0, g.n, 512).astype(np.int32)
    m, rep = B.b2sr_autotune(g.n, rp, ci, smp, sr, vk, keep_ratio=keep, trials=3)
    with m:
        oest, oth = oracle.sample_profile(g, smp)
        np.testing.assert_array_equal(np.array(rep["est_tiles"]), oth)
        best_est = min(rep["est_ratio"])
        tried = []
        for q, k in enumerate(KS):
            kept = keep <= 0 or rep["est_ratio"][q] <= keep * best_est
            assert (rep["tiles"][q] >= 0) == kept
            if kept:
                assert rep["tiles"][q] == len(oracle.b2sr(g, k)[1])
                assert rep["trial_us"][q][0] > 0
                for slot in range(2):
                    if rep["trial_us"][q][slot] > 0:
                        tried.append((rep["trial_us"][q][slot], k, slot))
        t, k, slot = min(tried)
        assert m.tile_dim == rep["tile_dim"] == k
        assert m.schedule == rep["schedule"]
        if rep["trial_us"][KS.index(k)][1] > 0:       # two schedules were tried
            assert rep["schedule"] == (1 if slot == 0 else 2)
        # the tuned handle computes the oracle's result
        if scheme == "bool":
            xb = graphs.random_bits(g.n, 0.1, seed=2)
            y = torch.empty(B.bitset_words(g.n), dtype=torch.int32, device="cuda")
            B.b2sr_spmv(m, sr, vk, to_dev(xb), vk, y)
            np.testing.assert_array_equal(to_np(y, np.uint32), oracle.spmv_bool(oracle.canonicalize(g), xb))
        else:
            x = np.random.default_rng(3).random(g.n).astype(np.float32)
            y = torch.empty(g.n, dtype=torch.float32, device="cuda")
            B.b2sr_spmv(m, sr, vk, to_dev(x), vk, y)
            if scheme == "plus":
                np.testing.assert_allclose(to_np(y).astype(np.float64),
                                           oracle.spmv_plus(oracle.canonicalize(g), x.astype(np.float64)),
                                           rtol=1e-5, atol=0)
            else:
                ref = oracle.spmv_minplus(oracle.canonicalize(g), x.astype(np.float64))
                np.testing.assert_array_equal(to_np(y), ref.astype(np.float32))


def test_autotune_rejects_bad_arguments(B):
    g = graphs.path(64)
    rp, ci = csr_dev(g)
    smp = np.arange(64, dtype=np.int32)
    with pytest.raises(B.B2SRError):
        B.b2sr_autotune(g.n, rp, ci, smp, B.BOOL_OR_AND, B.VEC_F32)          # no such scheme
    with pytest.raises(B.B2SRError):
        B.b2sr_autotune(g.n, rp, ci, smp, B.BOOL_OR_AND, B.VEC_BITS, keep_ratio=0.5)
    with pytest.raises(B.B2SRError):
        B.b2sr_autotune(g.n, rp, ci, smp, B.BOOL_OR_AND, B.VEC_BITS, trials=0)
    with B.b2sr_from_csr(g.n, rp, ci, 8) as m:
        with pytest.raises(B.B2SRError):
            B.b2sr_set_schedule(m, 3)
