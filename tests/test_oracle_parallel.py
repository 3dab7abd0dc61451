"""Pins for the oracle's parallel paths (og_new_par, og_count_par,
og_list_canonical_par), which the full-size parity tests and the CPU baseline
use.  Each is checked against what the mathematics fixes (brute force over all
triples, trace(A^3)/6 and diag(A^3)/2, closed forms) and against the serial
functions, at several thread counts (the result may not depend on them).
"""
import itertools

import numpy as np
import pytest

import graphgen as gg
import oracle


def adjacency(n, s, d):
    A = np.zeros((n, n), np.int64)
    keep = s != d
    A[s[keep], d[keep]] = 1
    A[d[keep], s[keep]] = 1
    return A


def random_pairs(n, num_edges, seed):
    rng = np.random.default_rng(seed)
    return rng.integers(0, n, num_edges).astype(np.int32), rng.integers(0, n, num_edges).astype(np.int32)


@pytest.mark.parametrize("n,num_edges,seed", [(30, 120, 0), (90, 1200, 1), (200, 6000, 2)])
@pytest.mark.parametrize("threads", [1, 3])
def test_brute_force(n, num_edges, seed, threads):
    s, d = random_pairs(n, num_edges, seed)
    A = adjacency(n, s, d)
    tri = [t for t in itertools.combinations(range(n), 3) if A[t[0], t[1]] and A[t[1], t[2]] and A[t[0], t[2]]]
    g = oracle.Graph(n, s, d, threads=threads)
    assert g.m == int(A.sum() // 2)
    T, t = g.count_per_vertex_par(threads)
    assert T == len(tri) == g.count_par(threads)
    ref_t = np.zeros(n, np.uint64)
    for x in tri:
        ref_t[list(x)] += 1
    assert np.array_equal(t, ref_t)
    # the canonical list holds exactly the brute-force set
    lst = g.list_canonical_par(oracle.ORDER_DESC, threads)
    assert sorted(tuple(sorted(r)) for r in lst.tolist()) == tri


@pytest.mark.parametrize("n,num_edges,seed", [(600, 12000, 10), (1500, 50000, 11)])
def test_trace_a_cubed(n, num_edges, seed):
    s, d = random_pairs(n, num_edges, seed)
    F = adjacency(n, s, d).astype(np.float64)
    A3 = np.rint(F @ F @ F).astype(np.int64)
    g = oracle.Graph(n, s, d, threads=0)
    T, t = g.count_per_vertex_par(0)
    assert 6 * T == int(np.trace(A3))
    assert np.array_equal(2 * t.astype(np.int64), np.diag(A3))


@pytest.mark.parametrize("case", ["k9", "wheel", "bip", "tri", "friend", "empty", "loops"])
def test_closed_forms(case):
    if case == "k9":
        (n, s, d), T = gg.complete(9), 84
    elif case == "wheel":
        (n, s, d), T = gg.wheel(13), 13
    elif case == "bip":
        (n, s, d), T = gg.random_bipartite(30, 40, 0.3, 5), 0
    elif case == "tri":
        (n, s, d), T = gg.complete_multipartite(3, 4, 5), 60
    elif case == "friend":
        (n, s, d), T = gg.friendship(7), 7
    elif case == "empty":
        (n, s, d), T = (6, np.zeros(0, np.int32), np.zeros(0, np.int32)), 0
    else:
        (n, s, d), T = (4, np.array([0, 1, 2], np.int32), np.array([0, 1, 2], np.int32)), 0
    g = oracle.Graph(n, s, d, threads=2)
    Tp, t = g.count_per_vertex_par(2)
    assert Tp == T and int(t.sum()) == 3 * T
    assert len(g.list_canonical_par(oracle.ORDER_DESC, 2)) == T


@pytest.mark.parametrize("order", [oracle.ORDER_DESC, oracle.ORDER_ASC, oracle.ORDER_DEGEN])
def test_equals_serial_on_rmat(order):
    n, s, d = gg.rmat_cfg(14, 9)
    ref = oracle.Graph(n, s, d)
    T, t = ref.count_per_vertex()
    off, adj = ref.csr()
    canon = ref.list_canonical(order)
    for threads in (1, 2, 7):
        g = oracle.Graph(n, s, d, threads=threads)
        o2, a2 = g.csr()
        assert np.array_equal(off, o2) and np.array_equal(adj, a2)
        Tp, tp = g.count_per_vertex_par(threads)
        assert Tp == T and np.array_equal(tp, t)
        assert np.array_equal(g.list_canonical_par(order, threads), canon)


def test_rejects_bad_ids():
    with pytest.raises(oracle.OracleError) as e:
        oracle.Graph(3, np.array([0, 3], np.int32), np.array([1, 1], np.int32), threads=2)
    assert e.value.status == oracle.ERR_RANGE

