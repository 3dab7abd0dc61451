"""Pins for the oracle: checks against what the paper and the mathematics fix,
never against the oracle itself.

* brute force over all vertex triples (n <= 200)
* trace(A^3)/6 and diag(A^3)/2 (exact int64 on CPU)
* closed forms: K_n, wheels, bipartite graphs, K_{a,b,c}, friendship graphs,
  cycles, stars, trees; sum of per-vertex counts = 3T
* Example 1 of Sec. 3.2 (tests/golden/example1.txt): the printed cost sums
* Algorithm 3 run literally (pure Python, global bitmap H) on small graphs:
  its output set equals the brute-force set (the correctness claim of
  Sec. 3.2) and its probe count equals the oracle's walk counter W
* eta / orientation invariants (Sec. 1, Sec. 2.2, footnote of Sec. 3.2)
"""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def adjacency(n, s, d):
    A = np.zeros((n, n), np.int64)
    for a, b in zip(s.tolist(), d.tolist()):
        if a != b:
            A[a, b] = A[b, a] = 1
    return A


def brute_force(n, A):
    tri = []
    for a, b, c in itertools.combinations(range(n), 3):
        if A[a, b] and A[b, c] and A[a, c]:
            tri.append((a, b, c))
    return tri


def random_graph(n, num_edges, seed):
    rng = np.random.default_rng(seed)
    s = rng.integers(0, n, num_edges).astype(np.int32)
    d = rng.integers(0, n, num_edges).astype(np.int32)
    return s, d


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("n,num_edges,seed", [(12, 30, 0), (40, 200, 1), (60, 900, 2),
                                              (120, 1500, 3), (200, 2500, 4), (200, 9000, 5)])
def test_brute_force_triples(n, num_edges, seed):
    s, d = random_graph(n, num_edges, seed)
    A = adjacency(n, s, d)
    tri = brute_force(n, A)
    g = oracle.Graph(n, s, d)
    assert g.m == int(A.sum() // 2)
    total, t = g.count_per_vertex()
    assert total == len(tri)
    ref_t = np.zeros(n, np.int64)
    for x in tri:
        for v in x:
            ref_t[v] += 1
    assert np.array_equal(t.astype(np.int64), ref_t)
    lst = g.list_ids()
    assert [tuple(r) for r in lst.tolist()] == tri  # id-sorted, lexicographic
    for v in range(0, n, 17):
        assert g.vertex_count(v) == ref_t[v]


# --------------------------------------------------------------- trace A^3
def a_cubed(A):
    """A^3 exactly: entries are at most n^2 < 2^53, so float64 BLAS is exact."""
    F = A.astype(np.float64)
    R = F @ F @ F
    assert R.max() < 2.0 ** 52
    return np.rint(R).astype(np.int64)


@pytest.mark.parametrize("n,num_edges,seed", [(500, 8000, 10), (2000, 60000, 11)])
def test_trace_a_cubed(n, num_edges, seed):
    s, d = random_graph(n, num_edges, seed)
    A3 = a_cubed(adjacency(n, s, d))
    g = oracle.Graph(n, s, d)
    total, t = g.count_per_vertex()
    assert 6 * total == int(np.trace(A3))
    assert np.array_equal(2 * t.astype(np.int64), np.diag(A3))


def test_trace_a_cubed_rmat():
    n, s, d = gg.rmat_cfg(10, seed=7)
    A3 = a_cubed(adjacency(n, s, d))
    total, t = oracle.Graph(n, s, d).count_per_vertex()
    assert 6 * total == int(np.trace(A3))
    assert np.array_equal(2 * t.astype(np.int64), np.diag(A3))


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("k", [3, 4, 5, 9, 30])
def test_complete(k):
    n, s, d = gg.complete(k)
    total, t = oracle.Graph(n, s, d).count_per_vertex()
    assert total == k * (k - 1) * (k - 2) // 6
    assert np.all(t == (k - 1) * (k - 2) // 2)


@pytest.mark.parametrize("rim", [4, 5, 8, 100])
def test_wheel(rim):
    n, s, d = gg.wheel(rim)
    total, t = oracle.Graph(n, s, d).count_per_vertex()
    assert total == rim
    assert t[0] == rim and np.all(t[1:] == 2)


def test_wheel_three_rim_is_k4():
    n, s, d = gg.wheel(3)  # rim 3 makes K_4
    assert oracle.Graph(n, s, d).count() == 4


@pytest.mark.parametrize("a,b,p,seed", [(10, 15, 0.5, 0), (50, 40, 0.3, 1), (5, 200, 0.9, 2)])
def test_bipartite_zero(a, b, p, seed):
    n, s, d = gg.random_bipartite(a, b, p, seed)
    total, t = oracle.Graph(n, s, d).count_per_vertex()
    assert total == 0 and not t.any()


@pytest.mark.parametrize("a,b,c", [(1, 1, 1), (2, 3, 4), (5, 6, 7)])
def test_tripartite(a, b, c):
    n, s, d = gg.complete_multipartite(a, b, c)
    total, t = oracle.Graph(n, s, d).count_per_vertex()
    assert total == a * b * c
    assert np.all(t[:a] == b * c) and np.all(t[a:a + b] == a * c) and np.all(t[a + b:] == a * b)


@pytest.mark.parametrize("k", [1, 2, 7, 50])
def test_friendship(k):
    n, s, d = gg.friendship(k)
    total, t = oracle.Graph(n, s, d).count_per_vertex()
    assert total == k and t[0] == k and np.all(t[1:] == 1)


def test_cycles_stars_trees():
    assert oracle.Graph(*gg.cycle(3)).count() == 1
    for k in (4, 5, 50):
        assert oracle.Graph(*gg.cycle(k)).count() == 0
    assert oracle.Graph(*gg.star(100)).count() == 0
    assert oracle.Graph(*gg.random_tree(300, 3)).count() == 0


def test_sum_per_vertex_is_three_t():
    n, s, d = gg.rmat_cfg(12, seed=3)
    total, t = oracle.Graph(n, s, d).count_per_vertex()
    assert int(t.sum()) == 3 * total and total > 0


# --------------------------------------------------------------- cleanup
def test_cleanup_invariance():
    s, d = random_graph(80, 600, 7)
    g0 = oracle.Graph(80, s, d)
    # loops, duplicates and reversed copies do not change the simple graph
    s2 = np.concatenate([s, d, s, np.arange(80, dtype=np.int32)])
    d2 = np.concatenate([d, s, d, np.arange(80, dtype=np.int32)])
    g1 = oracle.Graph(80, s2, d2)
    o0, a0 = g0.csr()
    o1, a1 = g1.csr()
    assert np.array_equal(o0, o1) and np.array_equal(a0, a1)
    assert g0.count_per_vertex()[0] == g1.count_per_vertex()[0]


def test_cleanup_rejects_bad_ids():
    with pytest.raises(oracle.OracleError) as e:
        oracle.Graph(10, np.array([0, 10], np.int32), np.array([1, 2], np.int32))
    assert e.value.status == oracle.ERR_RANGE
    with pytest.raises(oracle.OracleError):
        oracle.Graph(10, np.array([-1], np.int32), np.array([1], np.int32))


def test_empty_graphs():
    g = oracle.Graph(0, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.m == 0 and g.count() == 0
    g = oracle.Graph(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.count_per_vertex()[0] == 0
    g = oracle.Graph(3, np.array([1, 1], np.int32), np.array([1, 1], np.int32))
    assert g.m == 0


# ------------------------------------------------------------- Example 1
def load_example1():
    meta, edges, named = {}, [], []
    with open(os.path.join(GOLDEN, "example1.txt")) as f:
        for line in f:
            line = line.strip()
            if line.startswith("# n "):
                meta["n"] = int(line.split()[2])
            elif line.startswith("# expect "):
                k, v = line.split()[2:4]
                meta[k] = int(v)
            elif line.startswith("# edge "):
                named.append(tuple(int(x) for x in line.split()[2:6]))
            elif line and not line.startswith("#"):
                edges.append(tuple(int(x) for x in line.split()))
    e = np.array(edges, np.int32)
    return meta, e[:, 0], e[:, 1], named


def test_example1_costs():
    meta, s, d, named = load_example1()
    g = oracle.Graph(meta["n"], s, d)
    assert g.m == meta["m"]
    c = g.costs(oracle.ORDER_ASC)
    assert c["sum_deg_head"] == meta["sum_deg_head"]
    assert c["sum_min"] == meta["sum_min"]
    assert g.count() == meta["triangles"]
    # the orientation reproduces every named edge and its printed costs
    rank, perm, off, adj = g.orient(oracle.ORDER_ASC)
    outdeg = np.diff(off)
    heads = 0
    for u in range(g.n):
        for v in adj[off[u]:off[u + 1]]:
            heads += outdeg[v] > 0
    assert heads == meta["heads_with_outdeg"]
    for u, v, cost_kc, cost_min in named:
        ru, rv = rank[u], rank[v]
        assert ru < rv and rv in adj[off[ru]:off[ru + 1]]
        assert outdeg[rv] == cost_kc
        assert min(outdeg[ru], outdeg[rv]) == cost_min


# -------------------------------------------- Algorithm 3, run literally
def algorithm3(n, off, adj, clip=True, tail=False):
    """Algorithm 3 over an oriented CSR (rank space) with a global bitmap H.
    Ties of deg+ are broken by rank (footnote of the correctness argument);
    with clip the walk over N+(x) of a negative edge keeps the entries after
    the pivot, without it (as printed) it walks all of N+(x).  tail=True makes
    every edge <u,v> positive (u walks N+(v)): the node iterator of kClist,
    Algorithm 2, on the same orientation.
    Returns (triangles as rank triples, probes, per-pivot items, walks)."""
    outdeg = np.diff(off)
    ins = [[] for _ in range(n)]
    for x in range(n):
        for u in adj[off[x]:off[x + 1]]:
            ins[u].append(x)
    key = lambda x: (outdeg[x], x)
    H = np.zeros(n, bool)
    found, probes = [], 0
    items = np.zeros(n, np.int64)
    walks = np.zeros(n, np.int64)
    for u in range(n):
        Nu = adj[off[u]:off[u + 1]]
        H[Nu] = True
        for v in Nu:                          # positive edges <u,v>
            if tail or key(v) < key(u):
                items[u] += 1
                for w in adj[off[v]:off[v + 1]]:
                    probes += 1
                    walks[u] += 1
                    if H[w]:
                        found.append((u, v, w))
        for x in ins[u]:                      # negative edges <x,u>
            if not tail and key(x) < key(u):
                items[u] += 1
                for y in adj[off[x]:off[x + 1]]:
                    if clip and y <= u:
                        continue
                    probes += 1
                    walks[u] += 1
                    if H[y]:
                        found.append((x, u, y))
        H[Nu] = False
    return found, probes, items, walks


@pytest.mark.parametrize("order", [oracle.ORDER_DESC, oracle.ORDER_ASC])
@pytest.mark.parametrize("case", ["er", "rmat", "wheel", "k7", "example1"])
def test_algorithm3_literal(case, order):
    if case == "er":
        n = 150
        s, d = random_graph(n, 1400, 21)
    elif case == "rmat":
        n, s, d = gg.rmat_cfg(8, seed=5)
    elif case == "wheel":
        n, s, d = gg.wheel(9)
    elif case == "k7":
        n, s, d = gg.complete(7)
    else:
        meta, s, d, _ = load_example1()
        n = meta["n"]
    g = oracle.Graph(n, s, d)
    rank, perm, off, adj = g.orient(order)
    found, probes, items, walks = algorithm3(n, off, adj)
    # every triangle exactly once (Sec. 3.2 correctness)
    brute = brute_force(n, adjacency(n, s, d))
    assert len(found) == len(set(found)) == len(brute)
    assert sorted(tuple(sorted(perm[list(t)])) for t in found) == brute
    # every triple is an oriented triangle u<v<w in rank space
    assert all(a < b < c for a, b, c in found)
    c = g.costs(order)
    assert c["walk"] == probes
    assert probes <= c["sum_min"]
    oi, ow = g.work(order)
    assert np.array_equal(oi.astype(np.int64), items)
    assert np.array_equal(ow.astype(np.int64), walks)
    assert int(oi.sum()) == g.m


@pytest.mark.parametrize("rule", [1, 2])
@pytest.mark.parametrize("case", ["er", "rmat", "wheel", "example1"])
def test_algorithm3_rules_literal(case, rule):
    """Algorithm 3 as printed (rule 1, no clip) and the tail charging of
    kClist (rule 2): both find every triangle once; their probe counts equal
    the oracle's og_costs_noclip / sum of deg+(v) and og_work_rule per pivot."""
    if case == "er":
        n = 150
        s, d = random_graph(n, 1400, 22)
    elif case == "rmat":
        n, s, d = gg.rmat_cfg(8, seed=6)
    elif case == "wheel":
        n, s, d = gg.wheel(11)
    else:
        meta, s, d, _ = load_example1()
        n = meta["n"]
    g = oracle.Graph(n, s, d)
    for order in (oracle.ORDER_DESC, oracle.ORDER_ASC):
        rank, perm, off, adj = g.orient(order)
        found, probes, items, walks = algorithm3(n, off, adj, clip=False, tail=rule == 2)
        brute = brute_force(n, adjacency(n, s, d))
        assert sorted(tuple(sorted(perm[list(t)])) for t in found) == brute
        if rule == 1:
            assert probes == g.walk_noclip(order) >= g.costs(order)["walk"]
        else:
            assert probes == g.costs(order)["sum_deg_head"]
        oi, ow = g.work_rule(rule, order)
        assert np.array_equal(oi.astype(np.int64), items)
        assert np.array_equal(ow.astype(np.int64), walks)
        ci, cw = g.work_rule(0, order)
        wi, ww = g.work(order)
        assert np.array_equal(ci, wi) and np.array_equal(cw, ww)


def test_example1_walk():
    meta, s, d, _ = load_example1()
    c = oracle.Graph(meta["n"], s, d).costs(oracle.ORDER_ASC)
    # Per copy: <v3,v4> is positive and walks deg+(v4) = 2; the four edges into
    # the sinks are positive with deg+(sink) = 0; <v1,v3> and <v2,v4> are
    # negative edges whose clipped walk (entries of N+(v1) after v3) is empty.
    assert c["walk"] == 3 * 2 and c["positive"] == 3 * 5


# -------------------------------------------------- eta and orientation
@pytest.mark.parametrize("order", [oracle.ORDER_DESC, oracle.ORDER_ASC])
def test_eta_and_orientation_invariants(order):
    n, s, d = gg.rmat_cfg(11, seed=9)
    g = oracle.Graph(n, s, d)
    deg = g.degrees()
    rank, perm, off, adj = g.orient(order)
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert np.array_equal(rank[perm], np.arange(n))
    dp = deg[perm].astype(np.int64)
    steps = np.diff(dp)
    assert np.all(steps <= 0) if order == oracle.ORDER_DESC else np.all(steps >= 0)
    ties = steps == 0
    assert np.all(np.diff(perm)[ties] > 0)  # ties: smaller id first
    # every undirected edge once, from the earlier to the later eta position
    assert off[-1] == g.m
    src = np.repeat(np.arange(n), np.diff(off))
    assert np.all(src < adj)
    for u in range(0, n, 7):
        lst = adj[off[u]:off[u + 1]]
        assert np.all(np.diff(lst) > 0)
    und = set()
    goff, gadj = g.csr()
    for v in range(n):
        for w in gadj[goff[v]:goff[v + 1]]:
            if v < w:
                und.add((v, int(w)))
    ori = {tuple(sorted((int(perm[a]), int(perm[b])))) for a, b in zip(src, adj)}
    assert ori == und


def test_canonical_list_order():
    n, s, d = gg.rmat_cfg(9, seed=4)
    g = oracle.Graph(n, s, d)
    lst = g.list_canonical(oracle.ORDER_DESC)
    rank, _ = g.eta(oracle.ORDER_DESC)
    r = rank[lst]
    assert np.all(r[:, 0] < r[:, 1]) and np.all(r[:, 1] < r[:, 2])
    keys = [tuple(x) for x in r.tolist()]
    assert keys == sorted(keys) and len(set(keys)) == len(keys)
    ids = {tuple(sorted(t)) for t in lst.tolist()}
    assert ids == {tuple(t) for t in g.list_ids().tolist()}


# --------------------------------------------------- streaming sampler
def test_stream_vertex_counts():
    n, s, d = gg.rmat_cfg(10, seed=12)
    s = np.concatenate([s, d[:100]])
    d = np.concatenate([d, s[:100]])
    g = oracle.Graph(n, s, d)
    _, t = g.count_per_vertex()
    verts = np.array([0, 1, 5, int(np.argmax(t)), n - 1], np.int32)
    got = oracle.stream_vertex_counts(n, s, d, verts)
    assert np.array_equal(got, t[verts])


@pytest.mark.parametrize("order", [oracle.ORDER_DESC, oracle.ORDER_ASC])
def test_cost_identities(order):
    """Sec. 1 and Sec. 2.3: sum over <u,v> of deg+(v) equals sum over v of
    deg+(v) * deg-(v); the CF cost adds sum over u of deg+(u)^2."""
    n, s, d = gg.rmat_cfg(11, seed=13)
    g = oracle.Graph(n, s, d)
    rank, perm, off, adj = g.orient(order)
    outd = np.diff(off).astype(np.int64)
    ind = np.bincount(adj, minlength=n).astype(np.int64)
    c = g.costs(order)
    assert c["sum_deg_head"] == int((outd * ind).sum())
    assert c["sum_cf"] == int((outd * outd).sum()) + c["sum_deg_head"]
    assert c["walk"] <= c["sum_min"] <= c["sum_deg_head"]


# ------------------------------------------------------ degeneracy order
def _path(n):
    return n, np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32)


@pytest.mark.parametrize("case", ["er", "rmat10", "chunglu", "wheel", "k9", "bip"])
def test_degeneracy_levels_are_core_numbers(case):
    """The peeling's level of every vertex is its core number (networkx's
    core_number, an independent implementation); under the degeneracy order
    every vertex has at most its core number of later neighbours, and the
    largest out-degree is the degeneracy (Sec. 2.3: kClist orients by it)."""
    nx = pytest.importorskip("networkx")
    if case == "er":
        n = 300
        s, d = random_graph(n, 3000, 41)
    elif case == "rmat10":
        n, s, d = gg.rmat_cfg(10, seed=9)
    elif case == "chunglu":
        n = 2000
        s, d = gg.chunglu(n, 2.1, 12.0, seed=3)
    elif case == "wheel":
        n, s, d = gg.wheel(20)
    elif case == "k9":
        n, s, d = gg.complete(9)
    else:
        n, s, d = gg.random_bipartite(40, 50, 0.2, 2)
    g = oracle.Graph(n, s, d)
    G = nx.Graph()
    G.add_nodes_from(range(n))
    G.add_edges_from((int(a), int(b)) for a, b in zip(s, d) if a != b)
    core = nx.core_number(G)
    rnd, lvl = g.degeneracy()
    assert all(lvl[v] == core[v] for v in range(n))
    rank, perm, off, adj = g.orient(oracle.ORDER_DEGEN)
    outdeg = np.diff(off)
    assert np.all(outdeg[rank] <= lvl)
    assert outdeg.max(initial=0) == max(core.values(), default=0)
    # eta = (round, id)
    key = rnd.astype(np.int64) * n + np.arange(n)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    T, t = g.count_per_vertex()
    assert len(g.list_canonical(oracle.ORDER_DEGEN)) == T


def test_degeneracy_closed_forms():
    # a path peels from both ends, one vertex per end per round (level 1)
    n, s, d = _path(9)
    rnd, lvl = oracle.Graph(n, s, d).degeneracy()
    assert list(rnd) == [min(i, n - 1 - i) for i in range(n)] and set(lvl) == {1}
    # a star: the leaves in round 0, then the centre (degree 0 by then)
    n, s, d = gg.star(7)
    rnd, lvl = oracle.Graph(n, s, d).degeneracy()
    assert list(rnd) == [1] + [0] * 6 and list(lvl) == [1] * 7
    # K_n: nothing at levels below n-1, then everything in one round
    n, s, d = gg.complete(6)
    rnd, lvl = oracle.Graph(n, s, d).degeneracy()
    assert set(rnd) == {0} and set(lvl) == {5}
    # isolated vertices first (level 0), then a triangle
    rnd, lvl = oracle.Graph(5, np.array([2, 3, 4], np.int32), np.array([3, 4, 2], np.int32)).degeneracy()
    assert list(rnd) == [0, 0, 1, 1, 1] and list(lvl) == [0, 0, 2, 2, 2]
