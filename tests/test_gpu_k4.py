"""GPU parity at tile_dim 4, where the Boolean and count SpMVs and, under the
direct schedule, the unweighted 4-byte value schemes (plus-times, label min,
fp32 max) run on their own persistent kernel (each warp prefetches its next
chunk's tiles; a chunk inside one tile-row is joined by a butterfly instead of
the row walk), and the other value schemes on the general chunk kernel.  The
butterfly pairs lanes exactly as the chunk kernel's scan does, so the
four-column block (chunk kernel) still equals the single-column SpMV (tile_dim-4
kernel) bit for bit.

Every scheme is compared with the oracle on graphs with the tile patterns the
kernels treat apart: dense tiles (all sixteen bits set), short tile-rows of
multi-bit tiles, one row spanning many chunks (the cross-chunk join), empty
rows, a ragged n, and a masked level loop's all-masked chunks.  Bit-exact for
Boolean, integer, min, max and OR results; plus-times within 1e-5 relative
error of the fp64 oracle (the bound derived in test_gpu_spmv.py), and bitwise
reproducible from call to call.  The four-column PageRank block sums each
column exactly like the single-column SpMV."""
import numpy as np
import pytest
import torch

import oracle
from paper_2201_08560_gb300 import graphs
from tests.gpu_util import csr_dev, small_graphs, to_dev, to_np

pytestmark = pytest.mark.gpu

RTOL_F32 = 1e-5


def _graphs():
    out = [("rmat12", small_graphs()[0]), ("star20k", small_graphs()[2]), ("gaps", small_graphs()[4]),
           ("grid37x41", small_graphs()[3]), ("n1", small_graphs()[6])]
    # blocks of dense rows (multi-bit tiles) separated by short sparse rows
    dense = graphs.disjoint_union(graphs.complete(64), graphs.path(50), graphs.complete(37),
                                  graphs.random_symmetric(400, 0.3, seed=5), graphs.cycle(21))
    out.append(("dense_blocks", dense))
    out.append(("rmat13perm", graphs.rmat(13, 16, seed=7, permute_seed=8)))
    out.append(("directed", graphs.random_directed(1001, 0.02, seed=3)))
    return out


GRAPHS = _graphs()
IDS = [n for n, _ in GRAPHS]


@pytest.fixture(scope="module")
def B():
    from paper_2201_08560_gb300 import binding
    return binding


def _run_all(B, g, m):
    """Every SpMV scheme at tile_dim 4."""
    B.b2sr_set_schedule(m, 2)  # DIRECT
    n = g.n
    words = B.bitset_words(n)
    xb = graphs.random_bits(n, 0.1, seed=3)
    mask = graphs.random_bits(n, 0.5, seed=4)
    res = {}
    for tag, mk, comp in (("nomask", None, False), ("mask", mask, False), ("comp", mask, True)):
        y = torch.full((max(words, 1),), -1, dtype=torch.int32, device="cuda")
        B.b2sr_spmv(m, B.BOOL_OR_AND, B.VEC_BITS, to_dev(xb), B.VEC_BITS, y,
                    None if mk is None else to_dev(mk), comp)
        res["bool_" + tag] = to_np(y, np.uint32)[:words].copy()
        yc = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
        B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_BITS, to_dev(xb), B.VEC_I32, yc,
                    None if mk is None else to_dev(mk), comp)
        res["count_" + tag] = to_np(yc)[:n].copy()
    rng = np.random.default_rng(11)
    xf = rng.random(n).astype(np.float32)
    y = torch.full((max(n, 1),), float("nan"), dtype=torch.float32, device="cuda")
    B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(xf), B.VEC_F32, y)
    res["plus"] = to_np(y)[:n].copy()
    xm = (rng.integers(0, 50, n) / 4.0).astype(np.float32)
    B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_F32, to_dev(xm), B.VEC_F32, y)
    res["minplus"] = to_np(y)[:n].copy()
    B.b2sr_spmv(m, B.MAX_TIMES, B.VEC_F32, to_dev(xf), B.VEC_F32, y)
    res["max"] = to_np(y)[:n].copy()
    xl = rng.permutation(n).astype(np.int32)
    yi = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_I32, to_dev(xl), B.VEC_I32, yi)
    res["min_i32"] = to_np(yi)[:n].copy()
    X = rng.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64) & rng.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64)
    M = rng.integers(0, 2**63, n, dtype=np.int64).astype(np.uint64)
    Y = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    B.b2sr_spmm_bits64(m, to_dev(X), Y)
    res["or64"] = to_np(Y, np.uint64)[:n].copy()
    B.b2sr_spmm_bits64(m, to_dev(X), Y, to_dev(M), True)
    res["or64_comp"] = to_np(Y, np.uint64)[:n].copy()
    X4 = rng.random((n, 4)).astype(np.float32)
    Y4 = torch.full((max(n, 1), 4), float("nan"), dtype=torch.float32, device="cuda")
    B.b2sr_spmm_f32x4(m, to_dev(X4), Y4)
    res["plus4"] = to_np(Y4)[:n].copy()
    torch.cuda.synchronize()
    return res, dict(xb=xb, mask=mask, xf=xf, xm=xm, xl=xl, X=X, M=M, X4=X4)


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=IDS)
def test_k4_schemes_against_oracle(B, gi):
    name, g = GRAPHS[gi]
    rp, ci = csr_dev(g)
    cg = oracle.canonicalize(g)
    with B.b2sr_from_csr(g.n, rp, ci, 4) as m:
        got, inp = _run_all(B, g, m)
        for tag, mk, comp in (("nomask", None, False), ("mask", inp["mask"], False), ("comp", inp["mask"], True)):
            np.testing.assert_array_equal(got["bool_" + tag], oracle.spmv_bool(cg, inp["xb"], mk, comp))
            np.testing.assert_array_equal(got["count_" + tag], oracle.spmv_count(cg, inp["xb"], mk, comp))
        ref = oracle.spmv_plus(cg, inp["xf"].astype(np.float64))
        np.testing.assert_array_less(np.abs(got["plus"] - ref), RTOL_F32 * np.abs(ref) + 1e-30)
        np.testing.assert_array_equal(got["minplus"], oracle.spmv_minplus(cg, inp["xm"].astype(np.float64))
                                      .astype(np.float32))
        np.testing.assert_array_equal(got["max"], oracle.spmv_max(cg, inp["xf"].astype(np.float64)).astype(np.float32))
        np.testing.assert_array_equal(got["min_i32"], oracle.spmv_min_i32(cg, inp["xl"]))
        np.testing.assert_array_equal(got["or64"], oracle.spmm_or64(cg, inp["X"]))
        np.testing.assert_array_equal(got["or64_comp"], oracle.spmm_or64(cg, inp["X"], inp["M"], True))
        for b in range(4):
            refb = oracle.spmv_plus(cg, inp["X4"][:, b].astype(np.float64))
            np.testing.assert_array_less(np.abs(got["plus4"][:, b] - refb), RTOL_F32 * np.abs(refb) + 1e-30)
            yb = torch.empty(max(g.n, 1), dtype=torch.float32, device="cuda")
            B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(np.ascontiguousarray(inp["X4"][:, b])), B.VEC_F32, yb)
            np.testing.assert_array_equal(got["plus4"][:, b], to_np(yb)[: g.n])
        # bitwise reproducible
        again, _ = _run_all(B, g, m)
        for key in got:
            np.testing.assert_array_equal(again[key], got[key], err_msg=key)


def test_k4_masked_level_loop_skips_saturated_chunks(B):
    """A BFS level loop masks out the visited rows: chunks whose every row is
    visited read no tiles.  The multi-source BFS (OR64 with a complemented
    mask) and the single-source BFS (Boolean with a complemented mask) both
    pass through such chunks on R-MAT; levels equal the oracle's."""
    g = graphs.rmat(13, 16, seed=2)
    rp, ci = csr_dev(g)
    cg = oracle.canonicalize(g)
    srcs = [int(s) for s in graphs.sources(g, 20, seed=5)]
    with B.b2sr_from_csr(g.n, rp, ci, 4) as m:
        B.b2sr_set_schedule(m, 2)
        lv = B.b2sr_bfs_multi(m, srcs).cpu().numpy()
        for i, s in enumerate(srcs):
            ref = oracle.bfs(cg, s)
            np.testing.assert_array_equal(lv[i], ref)
            np.testing.assert_array_equal(B.b2sr_bfs(m, s).cpu().numpy(), ref)


@pytest.mark.parametrize("gi", range(len(GRAPHS)), ids=IDS)
def test_k4_value_schemes_with_masks(B, gi):
    """The value schemes the tile_dim-4 kernel runs (plus-times, fp32 max,
    label min) with a bit mask and its complement: masked-out rows get the
    semiring's identity, the others the unmasked result."""
    name, g = GRAPHS[gi]
    rp, ci = csr_dev(g)
    cg = oracle.canonicalize(g)
    n = g.n
    rng = np.random.default_rng(31)
    mask = graphs.random_bits(n, 0.4, seed=9)
    xf = rng.random(n).astype(np.float32)
    xl = rng.permutation(n).astype(np.int32)
    with B.b2sr_from_csr(n, rp, ci, 4) as m:
        B.b2sr_set_schedule(m, 2)  # DIRECT: the tile_dim-4 kernel
        y = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
        yi = torch.empty(max(n, 1), dtype=torch.int32, device="cuda")
        for comp in (False, True):
            B.b2sr_spmv(m, B.PLUS_TIMES, B.VEC_F32, to_dev(xf), B.VEC_F32, y, to_dev(mask), comp)
            ref = oracle.spmv_plus(cg, xf.astype(np.float64), mask, comp)
            got = to_np(y)[:n]
            np.testing.assert_array_less(np.abs(got - ref), RTOL_F32 * np.abs(ref) + 1e-30)
            B.b2sr_spmv(m, B.MAX_TIMES, B.VEC_F32, to_dev(xf), B.VEC_F32, y, to_dev(mask), comp)
            np.testing.assert_array_equal(to_np(y)[:n],
                                          oracle.spmv_max(cg, xf.astype(np.float64), mask, comp).astype(np.float32))
            B.b2sr_spmv(m, B.MIN_PLUS, B.VEC_I32, to_dev(xl), B.VEC_I32, yi, to_dev(mask), comp)
            np.testing.assert_array_equal(to_np(yi)[:n], oracle.spmv_min_i32(cg, xl, mask, comp))
