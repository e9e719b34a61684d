"""Oracle pins for the max-times semiring and the priority-ordered MIS and
colouring (Table 4: tropical max-times for MIS and graph colouring).  Each is
pinned by what the mathematics fixes rather than by retyping it: dense
algebra for the SpMV; independence, maximality and the first-in-priority
characterisation for the MIS; validity and closed forms for the colouring."""
import numpy as np
import pytest

import oracle
from paper_2201_08560_gb300 import graphs

pytestmark = pytest.mark.filterwarnings("ignore")


def dense(g):
    return graphs.to_dense(oracle.canonicalize(g))


def prio_for(n, seed):
    return np.random.default_rng(seed).permutation(n).astype(np.float64) + 1.0   # distinct


@pytest.mark.parametrize("seed", range(4))
def test_spmv_max_matches_dense(seed):
    g = graphs.random_directed(70, 0.08, seed)
    A = dense(g)
    x = np.random.default_rng(seed).normal(size=g.n)
    ref = np.where(A != 0, x[None, :], -np.inf).max(axis=1)
    np.testing.assert_array_equal(oracle.spmv_max(g, x), ref)
    mask = graphs.random_bits(g.n, 0.5, seed + 9)
    mb = graphs.unpack_bits(mask, g.n).astype(bool)
    np.testing.assert_array_equal(oracle.spmv_max(g, x, mask, False), np.where(mb, ref, -np.inf))
    np.testing.assert_array_equal(oracle.spmv_max(g, x, mask, True), np.where(~mb, ref, -np.inf))


def undirected_neighbours(g):
    A = dense(g) != 0
    A = A | A.T
    np.fill_diagonal(A, False)
    return A


GRAPHS = [graphs.rmat(9, 8, seed=1), graphs.grid2d(13, 17), graphs.star(40), graphs.complete(12),
          graphs.cycle(31), graphs.mycielski(6), graphs.from_dense(np.zeros((9, 9)))]


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("seed", range(3))
def test_mis_is_the_first_maximal_independent_set_in_priority_order(gi, seed):
    g = GRAPHS[gi]
    A = undirected_neighbours(g)
    pr = prio_for(g.n, seed)
    s = oracle.mis_greedy(g, pr).astype(bool)
    assert not (A & s[:, None] & s[None, :]).any()                    # independent
    assert (s | (A & s[None, :]).any(axis=1)).all()                   # maximal
    higher = A & (pr[None, :] > pr[:, None])                           # u higher than v
    # v is in the set exactly when no higher-priority neighbour is
    np.testing.assert_array_equal(s, ~(higher & s[None, :]).any(axis=1))


def test_mis_brute_force_tiny():
    """On graphs of at most 10 vertices: the lexicographically first maximal
    independent set in decreasing priority, found by enumerating subsets."""
    for seed in range(6):
        g = graphs.random_directed(9, 0.3, seed, self_loops=False)
        g = graphs.from_dense(((graphs.to_dense(g) + graphs.to_dense(g).T) != 0).astype(np.float64))
        A = undirected_neighbours(g)
        pr = prio_for(g.n, seed)
        order = np.argsort(-pr)
        best = None
        for bits in range(1 << g.n):
            s = np.array([(bits >> v) & 1 for v in range(g.n)], bool)
            if (A & s[:, None] & s[None, :]).any() or not (s | (A & s[None, :]).any(axis=1)).all():
                continue
            key = tuple(-int(s[v]) for v in order)               # prefer members early in the order
            if best is None or key < best[0]:
                best = (key, s)
        np.testing.assert_array_equal(oracle.mis_greedy(g, pr).astype(bool), best[1])


def test_mis_special_cases():
    n = 12
    pr = prio_for(n, 1)
    s = oracle.mis_greedy(graphs.complete(n), pr)
    assert s.sum() == 1 and s[np.argmax(pr)] == 1
    np.testing.assert_array_equal(oracle.mis_greedy(graphs.from_dense(np.zeros((n, n))), pr), np.ones(n))
    star = graphs.star(10)                                             # vertex 0 is the hub
    hub_high = np.arange(10, dtype=np.float64)[::-1] + 1.0
    np.testing.assert_array_equal(oracle.mis_greedy(star, hub_high), np.eye(10, dtype=np.int32)[0])
    hub_low = np.arange(10, dtype=np.float64) + 1.0
    np.testing.assert_array_equal(oracle.mis_greedy(star, hub_low), 1 - np.eye(10, dtype=np.int32)[0])
    path = graphs.path(9)                                              # priorities falling along the path
    np.testing.assert_array_equal(oracle.mis_greedy(path, 10.0 - np.arange(9.0)), (np.arange(9) % 2 == 0))


@pytest.mark.parametrize("gi", range(len(GRAPHS)))
@pytest.mark.parametrize("seed", range(3))
def test_colouring_is_valid_and_levelled(gi, seed):
    g = GRAPHS[gi]
    A = undirected_neighbours(g)
    pr = prio_for(g.n, seed)
    c = oracle.color_levels(g, pr)
    assert not (A & (c[:, None] == c[None, :])).any()                 # a proper colouring
    # colour 0 exactly at the local maxima; every colour k > 0 has a higher
    # neighbour of colour k-1 (so colours are as small as the levels allow)
    higher = A & (pr[None, :] > pr[:, None])
    np.testing.assert_array_equal(c == 0, ~higher.any(axis=1))
    for v in np.flatnonzero(c > 0):
        assert (c[higher[v]] == c[v] - 1).any()
    # and above every higher neighbour: together, 1 + the largest of theirs
    assert not (higher & (c[None, :] >= c[:, None])).any()


def test_colouring_closed_forms():
    n = 9
    pr = prio_for(n, 2)
    c = oracle.color_levels(graphs.complete(n), pr)
    np.testing.assert_array_equal(c, n - 1 - np.argsort(np.argsort(pr)))   # rank from the top
    np.testing.assert_array_equal(oracle.color_levels(graphs.from_dense(np.zeros((n, n))), pr), np.zeros(n))
    path = graphs.path(n)                                              # falling priorities: 0,1,2,...
    np.testing.assert_array_equal(oracle.color_levels(path, 100.0 - np.arange(n)), np.arange(n))
