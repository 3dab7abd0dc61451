"""Batched counting (aot_batch) against the oracle graph by graph, and the
autotuner (results never change)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import gpu_graph, u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aot():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available()
    import paper_2006_11494_gb300 as m
    return m


def make_batch(graphs):
    """graphs: list of (n, src, dst) with local ids -> device tensors."""
    import torch
    nv = np.array([g[0] for g in graphs], np.int32)
    counts = np.array([len(g[1]) for g in graphs], np.int64)
    ofs = np.zeros(len(graphs) + 1, np.int64)
    np.cumsum(counts, out=ofs[1:])
    src = np.concatenate([g[1] for g in graphs] + [np.zeros(0, np.int32)]).astype(np.int32)
    dst = np.concatenate([g[2] for g in graphs] + [np.zeros(0, np.int32)]).astype(np.int32)
    return (torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(),
            torch.from_numpy(ofs).cuda(), torch.from_numpy(nv).cuda(), nv, ofs)


def run_batch(aot, batch, route=0, stream=None):
    import torch
    src, dst, ofs, nv_d, nv, _ = batch
    G, N = len(nv), int(nv.sum())
    ws = torch.empty(aot.aot_batch_workspace_size(src.numel(), G, N), dtype=torch.uint8, device="cuda")
    tri = torch.empty(max(G, 1), dtype=torch.int64, device="cuda")
    vc = torch.empty(max(N, 1), dtype=torch.int64, device="cuda")
    aot.aot_batch(src, dst, ofs, nv_d, route, tri, vc, ws, N, stream)
    return u64(tri[:G]), u64(vc[:N])


def small_graphs():
    out = []
    for i in range(30):
        n = 256 + 64 * i
        s, d = gg.chunglu(n, 2.5, 4.0 + 2 * i, seed=500 + i)
        out.append((n, s, d))
    out.append(gg.complete(5))
    out.append(gg.wheel(50))
    out.append((7, np.zeros(0, np.int32), np.zeros(0, np.int32)))          # no edges
    out.append((3, np.array([1, 2], np.int32), np.array([1, 2], np.int32)))  # loops only
    out.append((1, np.zeros(0, np.int32), np.zeros(0, np.int32)))          # one vertex
    out.append(gg.complete_multipartite(3, 4, 5))
    return out


def check_against_oracle(graphs, tri, vc, idx=None):
    voff = np.concatenate([[0], np.cumsum([g[0] for g in graphs])])
    for i in (range(len(graphs)) if idx is None else idx):
        n, s, d = graphs[i]
        T, t = oracle.Graph(n, s, d).count_per_vertex()
        assert tri[i] == T, i
        assert np.array_equal(vc[voff[i]:voff[i + 1]], t), i


@pytest.mark.parametrize("route", ["PLAIN", "RANDOM", "BSEARCH"])
def test_small_batch_matches_oracle(aot, route):
    import torch
    graphs = small_graphs()
    batch = make_batch(graphs)
    tri, vc = run_batch(aot, batch, getattr(aot, "ROUTE_" + route), torch.cuda.Stream())
    check_against_oracle(graphs, tri, vc)


def test_batch_on_default_and_side_streams(aot):
    import torch
    graphs = small_graphs()[:12]
    batch = make_batch(graphs)
    a = run_batch(aot, batch, 0, None)                  # launched directly
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        b = run_batch(aot, batch, 0, st)                # captured into a CUDA graph
    st.synchronize()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    check_against_oracle(graphs, *a)


def test_batch_graph_reused_across_calls(aot):
    """Several batches in a row on one stream: the thread's instantiated
    counting graph is updated in place (same kernels) or rebuilt (different
    ones); every result matches the oracle."""
    import torch
    st = torch.cuda.Stream()
    graphs = small_graphs()
    for part in (graphs[:10], graphs[10:20], graphs[:10], graphs[20:], graphs):
        batch = make_batch(part)
        tri, vc = run_batch(aot, batch, 0, st)
        check_against_oracle(part, tri, vc)


def test_batch_rejects_bad_input(aot):
    import torch
    graphs = [gg.complete(4), gg.complete(5)]
    src, dst, ofs, nv_d, nv, o = make_batch(graphs)
    bad = src.clone()
    bad[0] = 4                                           # vertex 4 does not exist in K_4
    with pytest.raises(aot.AotError) as e:
        run_batch(aot, (bad, dst, ofs, nv_d, nv, o))
    assert e.value.status == aot.ERR_VERTEX_RANGE
    ofs_bad = ofs.clone()
    ofs_bad[1] = ofs[2] + 1                              # offsets not monotone / not ending at E
    with pytest.raises(aot.AotError) as e:
        run_batch(aot, (src, dst, ofs_bad, nv_d, nv, o))
    assert e.value.status == aot.ERR_INVALID_ARG
    tri, vc = run_batch(aot, (src, dst, ofs, nv_d, nv, o))  # still usable
    assert list(tri) == [4, 10]


def oracle_counts_threaded(graphs):
    """(T, t) of every graph by the oracle's CF edge iterator (one thread per
    graph; pinned to the serial oracle in test_oracle_parallel.py), graphs
    spread over host threads (the oracle's C calls release the GIL; no process
    is forked)."""
    import concurrent.futures as cf

    def one(g):
        return oracle.Graph(*g, threads=1).count_per_vertex_par(1)
    with cf.ThreadPoolExecutor(max_workers=oracle.host_threads()) as ex:
        return list(ex.map(one, graphs))


def test_batch_of_4096_chunglu_graphs(aot):
    """4096 Chung-Lu graphs (n log-uniform in [256, 65536], mean degree
    uniform in [4, 64], gamma 2.5), with the tuning the batch autotuner picks
    on their union graph: every graph's T and t(v) against the oracle."""
    import torch
    nv, ofs, s, d = gg.batch(4096)
    batch = (torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), torch.from_numpy(ofs).cuda(),
             torch.from_numpy(nv).cuda(), nv, ofs)
    G, N = len(nv), int(nv.sum())
    ws = torch.empty(aot.aot_batch_workspace_size(len(s), G, N), dtype=torch.uint8, device="cuda")
    best, ms = aot.aot_batch_tune(batch[0], batch[1], batch[2], batch[3], ws, N)
    assert ms > 0 and best.hub_mode == 0
    old = aot.aot_get_default_tuning()
    try:
        aot.aot_set_default_tuning(best)
        tri, vc = run_batch(aot, batch, 0, torch.cuda.Stream())
    finally:
        aot.aot_set_default_tuning(old)
    graphs = [(int(nv[i]), s[ofs[i]:ofs[i + 1]], d[ofs[i]:ofs[i + 1]]) for i in range(len(nv))]
    ref = oracle_counts_threaded(graphs)
    voff = np.concatenate([[0], np.cumsum(nv.astype(np.int64))])
    for i, (T, t) in enumerate(ref):
        assert tri[i] == T, i
        assert np.array_equal(vc[voff[i]:voff[i + 1]], t), i


def test_autotuner_keeps_results(aot):
    n, s, d = gg.rmat_cfg(14, 41)
    g = gpu_graph(n, s, d)
    T0 = g.count()
    _, t0 = g.count_per_vertex()
    for mode in (0, 1):
        t, ms = aot.aot_tune(g.handle, mode, 1)
        assert ms > 0
        cur = aot.aot_graph_get_tuning(g.handle)
        assert cur.as_dict() == t.as_dict()
        assert g.count() == T0
        _, t1 = g.count_per_vertex()
        assert np.array_equal(u64(t1), u64(t0))
    # the default tuning is picked up by later graphs
    old = aot.aot_get_default_tuning()
    try:
        aot.aot_set_default_tuning(t)
        g2 = gpu_graph(n, s, d)
        assert aot.aot_graph_get_tuning(g2.handle).as_dict() == t.as_dict()
        assert g2.count() == T0
    finally:
        aot.aot_set_default_tuning(old)
