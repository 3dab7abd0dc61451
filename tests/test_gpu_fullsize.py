"""Full-size workloads against the oracle.

* R-MAT scale 20: m and W against the oracle; T and EVERY t(v) against the
  oracle's parallel edge iterator; the full canonical list, streamed in
  chunks of 2^26 triangles, element by element against the oracle's
  canonical list.
* R-MAT scale 24: T and EVERY t(v) against the oracle's parallel edge
  iterator; the list streamed in chunks of 2^28 triangles (10.3 G triangles,
  123 GB: too large to hold on the host), checked for canonical order on the
  GPU, for its length T, and on sampled triangles.
* R-MAT scale 27 and Chung-Lu 2^27 (gamma 2.1, mean degree 32): count and
  per-vertex counts; sampled t(v) from the raw edge list; the learned route
  and the global-bitmap hub path agree.  The oracle's full count at this size
  needs ~15 GB of host memory per graph and tens of minutes of host time, so
  these two stay sampled.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import u64

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def aot():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    import paper_2006_11494_gb300 as m
    return m


def edge_keys(s, d):
    """Sorted distinct undirected edges of a raw pair list as uint64 keys
    (sort, then drop repeats: far faster than np.unique at 2^28 keys)."""
    a = np.minimum(s, d).astype(np.uint64)
    b = np.maximum(s, d).astype(np.uint64)
    keep = a != b
    k = np.sort((a[keep] << np.uint64(32)) | b[keep])
    if len(k) == 0:
        return k
    first = np.empty(len(k), bool)
    first[0] = True
    np.not_equal(k[1:], k[:-1], out=first[1:])
    return k[first]


def eta_ranks(n, keys):
    """Degree non-increasing, ties by smaller id (plain definition)."""
    deg = np.bincount((keys >> np.uint64(32)).astype(np.int64), minlength=n) + \
        np.bincount((keys & np.uint64(0xffffffff)).astype(np.int64), minlength=n)
    order = np.lexsort((np.arange(n), -deg))
    rank = np.empty(n, np.int64)
    rank[order] = np.arange(n)
    return rank, deg


def has_edges(keys, x, y):
    a = np.minimum(x, y).astype(np.uint64)
    b = np.maximum(x, y).astype(np.uint64)
    q = (a << np.uint64(32)) | b
    pos = np.searchsorted(keys, q)
    pos = np.minimum(pos, len(keys) - 1)
    return keys[pos] == q


class ListChecker:
    """Canonical order of streamed chunks, checked on the GPU: ranks strictly
    increasing inside a triangle and lexicographically across triangles."""

    def __init__(self, rank):
        import torch
        self.rank = torch.from_numpy(rank).cuda()
        self.last = None
        self.total = 0

    def feed(self, tri):
        import torch
        r = self.rank[tri.long()]
        assert bool((r[:, 0] < r[:, 1]).all()) and bool((r[:, 1] < r[:, 2]).all())
        if self.last is not None:
            r = torch.cat([self.last[None], r])
        a, b = r[:-1], r[1:]
        gt = (b[:, 0] > a[:, 0]) | ((b[:, 0] == a[:, 0]) & ((b[:, 1] > a[:, 1]) |
                                                           ((b[:, 1] == a[:, 1]) & (b[:, 2] > a[:, 2]))))
        assert bool(gt.all())
        self.last = r[-1].clone()
        self.total += tri.shape[0]


def stream_list(aot, g, cap, rank, keys, samples_per_chunk, rng):
    import torch
    out = torch.empty(3 * cap, dtype=torch.int32, device="cuda")
    chk = ListChecker(rank)
    cursor = 0
    while True:
        k, nxt = aot.aot_list(g.handle, aot.ROUTE_PLAIN, cursor, out, cap)
        if k == 0:
            break
        tri = out[: 3 * k].view(-1, 3)
        chk.feed(tri)
        idx = rng.integers(0, k, samples_per_chunk)
        t = tri[torch.from_numpy(idx).cuda()].cpu().numpy()
        assert has_edges(keys, t[:, 0], t[:, 1]).all()
        assert has_edges(keys, t[:, 1], t[:, 2]).all()
        assert has_edges(keys, t[:, 0], t[:, 2]).all()
        cursor = nxt
        if k < cap:
            break
    return chk.total


def orient(aot, n, s, d, flags=0):
    import torch
    return aot.OrientedGraph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n, flags)


def stream_list_exact(aot, g, cap, ref_list):
    """Stream the GPU list in chunks and compare each chunk with the oracle's
    canonical list element by element."""
    import torch
    out = torch.empty(3 * cap, dtype=torch.int32, device="cuda")
    cursor = 0
    while True:
        k, nxt = aot.aot_list(g.handle, aot.ROUTE_PLAIN, cursor, out, cap)
        if k == 0:
            break
        got = out[: 3 * k].view(-1, 3).cpu().numpy()
        assert np.array_equal(got, ref_list[cursor:cursor + k]), cursor
        cursor = nxt
    return cursor


def test_rmat20_full_size(aot):
    n, s, d = gg.rmat_cfg(20, 2)
    ref = oracle.Graph(n, s, d, threads=0)
    g = orient(aot, n, s, d)
    assert g.m == ref.m
    assert g.info["W"] == ref.costs()["walk"]
    T_ref, t_ref = ref.count_per_vertex_par()
    T = g.count()
    T2, t = g.count_per_vertex()
    assert T == T2 == T_ref
    assert np.array_equal(u64(t), t_ref)
    del t
    ref_list = ref.list_canonical_par(oracle.ORDER_DESC)
    assert len(ref_list) == T_ref
    assert stream_list_exact(aot, g, 1 << 26, ref_list) == T_ref


def test_rmat20_variant_work_counters(aot):
    """Config 2: the work counters of AOT's orders and ablations and of the
    kClist / CF charging equal the oracle's cost counters exactly (Sec. 2.2,
    2.3, 3.2), and every variant counts the same triangles."""
    import torch
    n, s, d = gg.rmat_cfg(20, 2)
    ref = oracle.Graph(n, s, d, threads=0)
    T_ref = ref.count_par()
    src, dst = torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda()
    cost = {o: ref.costs(o) for o in (oracle.ORDER_DESC, oracle.ORDER_ASC, oracle.ORDER_DEGEN)}
    cases = [
        (0, "walk", cost[oracle.ORDER_DESC]["walk"]),
        (aot.ETA_DEG_ASC, "walk", cost[oracle.ORDER_ASC]["walk"]),
        (aot.ETA_DEGENERACY, "walk", cost[oracle.ORDER_DEGEN]["walk"]),
        (aot.FLAG_NO_CLIP, "walk", ref.walk_noclip(oracle.ORDER_DESC)),
        (aot.FLAG_LOCAL_RANDOM, "walk", ref.walk_noclip(oracle.ORDER_DESC)),
        (aot.FLAG_TAIL_PIVOT, "walk", cost[oracle.ORDER_DESC]["sum_deg_head"]),
        (aot.ETA_DEGENERACY | aot.FLAG_TAIL_PIVOT, "walk", cost[oracle.ORDER_DEGEN]["sum_deg_head"]),
        (aot.ETA_DEG_ASC | aot.FLAG_TAIL_PIVOT, "merge", cost[oracle.ORDER_ASC]["sum_cf"]),
    ]
    for flags, key, want in cases:
        g = aot.OrientedGraph(src, dst, n, flags | aot.FLAG_NO_LIST)
        assert aot.aot_graph_costs(g.handle)[key] == want, (flags, key)
        route = aot.ROUTE_MERGE if key == "merge" else aot.ROUTE_PLAIN
        assert g.count(route) == T_ref, flags
        g.close()


def test_rmat24_full_counts_and_streamed_listing(aot):
    rng = np.random.default_rng(24)
    n, s, d = gg.rmat_cfg(24, 3)
    g = orient(aot, n, s, d, aot.FLAG_NO_LIST)
    ref = oracle.Graph(n, s, d, threads=0)
    assert g.m == ref.m
    T_ref, t_ref = ref.count_per_vertex_par()
    del ref
    T = g.count()
    T2, t = g.count_per_vertex()
    assert T == T2 == T_ref
    assert np.array_equal(u64(t), t_ref)
    del t, t_ref
    g.close()
    keys = edge_keys(s, d)
    rank, _ = eta_ranks(n, keys)
    g = orient(aot, n, s, d)  # with the listing arrays
    assert stream_list(aot, g, 1 << 28, rank, keys, 300, rng) == T


@pytest.mark.parametrize("which", ["rmat27", "chunglu27"])
def test_two_billion_pair_graphs(aot, which):
    import torch
    from paper_2006_11494_gb300 import router
    rng = np.random.default_rng(27)
    if which == "rmat27":
        n, s, d = gg.rmat_cfg(27, 4)
    else:
        n = 1 << 27
        s, d = gg.chunglu(n, 2.1, 32.0, seed=5)
    g = orient(aot, n, s, d, aot.FLAG_NO_LIST)
    assert g.m > 1_000_000_000
    T = g.count()
    T2, t = g.count_per_vertex()
    t = u64(t)
    assert T == T2 and int(t.sum()) == 3 * T and T > 0
    deg_sample = rng.choice(n, 200000, replace=False).astype(np.int32)
    tv = t[deg_sample]
    pick = np.concatenate([deg_sample[np.nonzero(tv)[0][:2]], deg_sample[:1]]).astype(np.int32)
    assert np.array_equal(oracle.stream_vertex_counts(n, s, d, pick), t[pick])
    model = router.load()
    assert model is not None
    aot.aot_graph_set_router(g.handle, model)
    assert g.count(aot.ROUTE_LEARNED) == T
    g.set_tuning(hub_mode=1)  # hubs on the multi-CTA global-bitmap path
    assert g.count() == T
