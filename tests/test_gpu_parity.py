"""GPU parity: the CUDA path through the C ABI against the oracle, element by
element, on seeded inputs (bit-exact: every output here is an integer)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from helpers import gpu_graph, to_dev, u64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"


def check_full(n, s, d, flags=0, order=oracle.ORDER_DESC, listing=True, tuning=None, chunk=1 << 20):
    import paper_2006_11494_gb300 as aot
    ref = oracle.Graph(n, s, d)
    g = gpu_graph(n, s, d, flags)
    if tuning:
        g.set_tuning(**tuning)
    assert g.m == ref.m
    T_ref, t_ref = ref.count_per_vertex()
    assert g.count() == T_ref
    T, t = g.count_per_vertex()
    assert T == T_ref
    assert np.array_equal(u64(t), t_ref)
    if listing:
        lst = g.list(chunk=chunk).cpu().numpy()
        assert np.array_equal(lst, ref.list_canonical(order))
    for r in (aot.ROUTE_PROBE, aot.ROUTE_MERGE, aot.ROUTE_BSEARCH, aot.ROUTE_RANDOM):
        assert g.count(r) == T_ref, r
    return g, ref


ROUTES = ["PLAIN", "PROBE", "MERGE", "BSEARCH", "RANDOM"]


def check_routes(n, s, d, tuning=None):
    """Every route gives the same count, per-vertex counts and canonical list."""
    import paper_2006_11494_gb300 as aot
    ref = oracle.Graph(n, s, d)
    T_ref, t_ref = ref.count_per_vertex()
    lst_ref = ref.list_canonical()
    for name in ROUTES:
        r = getattr(aot, "ROUTE_" + name)
        g = gpu_graph(n, s, d)
        if tuning:
            g.set_tuning(**tuning)
        assert g.count(r) == T_ref, name
        T, t = g.count_per_vertex(r)
        assert T == T_ref and np.array_equal(u64(t), t_ref), name
        lst = g.list(r, chunk=max(1, len(lst_ref) // 3 + 1)).cpu().numpy()
        assert np.array_equal(lst, lst_ref), name


# ------------------------------------------------------------ closed forms
@pytest.mark.parametrize("case", ["k3", "k4", "k10", "k70", "w4", "w50", "w300", "bip", "tri",
                                  "f1", "f30", "c3", "c100", "star", "tree"])
def test_closed_forms(case):
    make = {
        "k3": lambda: gg.complete(3), "k4": lambda: gg.complete(4), "k10": lambda: gg.complete(10),
        "k70": lambda: gg.complete(70), "w4": lambda: gg.wheel(4), "w50": lambda: gg.wheel(50),
        "w300": lambda: gg.wheel(300), "bip": lambda: gg.random_bipartite(40, 70, 0.3, 1),
        "tri": lambda: gg.complete_multipartite(5, 6, 7), "f1": lambda: gg.friendship(1),
        "f30": lambda: gg.friendship(30), "c3": lambda: gg.cycle(3), "c100": lambda: gg.cycle(100),
        "star": lambda: gg.star(1000), "tree": lambda: gg.random_tree(500, 2),
    }[case]
    n, s, d = make()
    check_full(n, s, d)


# ------------------------------------------- ER, n = 16384, 262144 pairs
def test_er_16k_full_parity_and_orientation():
    n, s, d = gg.er_16k()
    g, ref = check_full(n, s, d)
    rank, perm, off, adj = ref.orient(oracle.ORDER_DESC)
    ex = g.export()
    assert np.array_equal(ex["perm"].cpu().numpy(), perm)
    assert np.array_equal(ex["rank"].cpu().numpy(), rank)
    assert np.array_equal(ex["out_off"].cpu().numpy().astype(np.int64), off)
    assert np.array_equal(ex["out_adj"].cpu().numpy(), adj)
    items, walk = ref.work(oracle.ORDER_DESC)
    assert np.array_equal(ex["items"].cpu().numpy().astype(np.uint32), items)
    assert np.array_equal(ex["walk"].cpu().numpy().astype(np.uint64), walk)
    c = ref.costs(oracle.ORDER_DESC)
    assert g.info["W"] == c["walk"]
    outd = np.diff(off)
    assert g.info["S"] == int(outd[items > 0].sum())
    assert g.info["max_outdeg"] == int(outd.max())


# ------------------------------------------------------- R-MAT, small scales
@pytest.mark.parametrize("scale,seed", [(8, 1), (10, 2), (12, 3), (14, 2)])
def test_rmat_full_parity(scale, seed):
    n, s, d = gg.rmat_cfg(scale, seed)
    g, ref = check_full(n, s, d)
    assert g.info["W"] == ref.costs()["walk"]


def test_chunglu_full_parity():
    s, d = gg.chunglu(1 << 13, 2.1, 24.0, seed=5)
    check_full(1 << 13, s, d)


@pytest.mark.parametrize("tuning", [
    dict(warp_max_outdeg=0, cta_max_outdeg=0, hub_bitmaps=1),      # everything on the hub path
    dict(warp_max_outdeg=0, cta_max_outdeg=0, hub_bitmaps=32),
    dict(warp_max_outdeg=64, cta_max_outdeg=64),                   # warp + hub
    dict(warp_max_outdeg=1, cta_max_outdeg=8192, cta_threads=128),  # almost all CTA
    dict(warp_max_outdeg=1, cta_max_outdeg=8192, cta_threads=32),   # the CTA bin a warp per pivot
    dict(warp_max_outdeg=16, cta_max_outdeg=512, cta_threads=32),
    dict(warp_max_outdeg=16, cta_max_outdeg=256, cta_threads=1024, hub_bitmaps=3),
    dict(warp_max_outdeg=0, cta_max_outdeg=0, hub_mode=1, hub_bitmaps=7),  # global bitmaps
    dict(warp_max_outdeg=8, cta_max_outdeg=64, hub_mode=0, seg_bits=1024),  # many segments
    dict(warp_max_outdeg=0, cta_max_outdeg=0, hub_mode=0, seg_bits=4096),
    dict(warp_max_outdeg=0, cta_max_outdeg=0, seg_wide=0),          # every warp walk in 256-entry rounds
    dict(warp_max_outdeg=0, cta_max_outdeg=0, seg_wide=1 << 30),    # every warp walk in 128-entry rounds
    dict(warp_max_outdeg=8, cta_max_outdeg=64, seg_bits=1024, seg_long=0, seg_wide=0),  # all warp-wide
    dict(warp_max_outdeg=8, cta_max_outdeg=64, seg_bits=2048, seg_long=1 << 30),        # all per-thread
    # every pivot on the bitmap path with 1024-rank segments: the per-pivot
    # segment bounds do not fit their scratch, so each segment end is searched
    dict(warp_max_outdeg=0, cta_max_outdeg=0, seg_bits=1024),
    # later segments: long items with few entries left walked per thread
    dict(warp_max_outdeg=8, cta_max_outdeg=64, seg_bits=2048, seg_long=0, seg_tail=1 << 20),
    dict(warp_max_outdeg=0, cta_max_outdeg=0, seg_bits=1024, seg_long=64, seg_tail=200),
    # smaller CTAs of the segmented bitmap kernel (two per SM)
    dict(warp_max_outdeg=0, cta_max_outdeg=0, seg_threads=512, seg_bits=524288),
    dict(warp_max_outdeg=8, cta_max_outdeg=64, seg_threads=256, seg_bits=2048, seg_tail=100),
    # pivot tails past the first segment in one hashed pass: never, up to
    # 3/8 of the table (32 to 128 slots here), up to the whole table (most
    # builds fail and fall back to the segments), or for some pivots only;
    # warp-wide or per-thread walks through the tail table
    dict(warp_max_outdeg=0, cta_max_outdeg=0, seg_bits=1024, seg_hash=0),
    dict(warp_max_outdeg=0, cta_max_outdeg=0, seg_bits=1024, seg_hash=12),
    dict(warp_max_outdeg=0, cta_max_outdeg=0, seg_bits=4096, seg_hash=1 << 30),
    dict(warp_max_outdeg=8, cta_max_outdeg=64, seg_bits=2048, seg_hash=5),
    dict(warp_max_outdeg=8, cta_max_outdeg=64, seg_bits=1024, seg_long=0, seg_wide=0, seg_tail=0),
    dict(warp_max_outdeg=8, cta_max_outdeg=64, seg_bits=1024, seg_long=1 << 30, seg_hash=1 << 30),
    # walked-list tiles: none, several (clamped when most pivots are hubs)
    dict(tile_bits=0),
    dict(warp_max_outdeg=64, cta_max_outdeg=64, tile_bits=16),
    dict(warp_max_outdeg=0, cta_max_outdeg=0, tile_bits=16),
])
def test_every_bin_gives_the_same_answer(tuning):
    n, s, d = gg.rmat_cfg(13, 7)
    check_full(n, s, d, tuning=tuning)


@pytest.mark.parametrize("tile_bits,seg_bits,seg_tail,seg_hash", [
    (16, 1572864, 0, 12288), (17, 4096, 0, 12288), (0, 4096, 0, 12288), (0, 4096, 512, 12288),
    (16, 8192, 1 << 30, 12288), (0, 4096, 128, 0), (0, 16384, 128, 192), (0, 16384, 128, 100),
    (0, 16384, 128, 1 << 30)])
def test_walk_tiles(tile_bits, seg_bits, seg_tail, seg_hash):
    """Hub tasks handed out tile by tile of the walked out-lists (16 tiles of
    2^16 entries at R-MAT scale 16), with one or many bitmap segments, and the
    pivot tails past the first segment swept or hashed (tables of up to 512
    slots at 16384-rank segments)."""
    n, s, d = gg.rmat_cfg(16, 5)
    check_full(n, s, d, tuning=dict(warp_max_outdeg=32, cta_max_outdeg=128, tile_bits=tile_bits,
                                    seg_bits=seg_bits, seg_tail=seg_tail, seg_hash=seg_hash))


@pytest.mark.parametrize("case", ["rmat12", "er", "wheel", "k40", "chunglu"])
def test_routes_are_invisible_in_the_output(case):
    if case == "rmat12":
        n, s, d = gg.rmat_cfg(12, 21)
    elif case == "er":
        n = 3000
        s, d = gg.er(n, 40000, seed=4)
    elif case == "wheel":
        n, s, d = gg.wheel(5000)
    elif case == "k40":
        n, s, d = gg.complete(40)
    else:
        n = 1 << 12
        s, d = gg.chunglu(n, 2.1, 20.0, seed=8)
    check_routes(n, s, d)


def test_routes_with_every_bin():
    n, s, d = gg.rmat_cfg(12, 22)
    check_routes(n, s, d, tuning=dict(warp_max_outdeg=16, cta_max_outdeg=128, seg_bits=2048))


def test_asc_order_orientation_and_parity():
    import paper_2006_11494_gb300 as aot
    n, s, d = gg.rmat_cfg(12, 5)
    g, ref = check_full(n, s, d, flags=aot.ETA_DEG_ASC, order=oracle.ORDER_ASC)
    rank, perm, off, adj = ref.orient(oracle.ORDER_ASC)
    ex = g.export()
    assert np.array_equal(ex["perm"].cpu().numpy(), perm)
    assert np.array_equal(ex["out_adj"].cpu().numpy(), adj)
    assert g.info["W"] == ref.costs(oracle.ORDER_ASC)["walk"]


@pytest.mark.parametrize("order", [oracle.ORDER_DESC, oracle.ORDER_ASC])
@pytest.mark.parametrize("case", ["rmat", "chunglu"])
def test_no_clip_and_tail_pivot(case, order):
    """Algorithm 3 as printed (no suffix clip) and the tail charging of
    kClist / CF: identical counts, per-vertex counts and canonical list; the
    work counters equal the oracle's (W without the clip; sum of deg+(v) for
    the tail rule, and sum of deg+(u) + deg+(v), CF's merge work, for its
    merge route); per-pivot items and walks equal og_work_rule."""
    import paper_2006_11494_gb300 as aot
    if case == "rmat":
        n, s, d = gg.rmat_cfg(13, 4)
    else:
        n = 1 << 12
        s, d = gg.chunglu(n, 2.1, 24.0, seed=31)
    eta = aot.ETA_DEG_ASC if order == oracle.ORDER_ASC else 0
    ref = oracle.Graph(n, s, d)
    c = ref.costs(order)
    for flag, rule in ((aot.FLAG_NO_CLIP, 1), (aot.FLAG_TAIL_PIVOT, 2)):
        g, _ = check_full(n, s, d, flags=eta | flag, order=order)
        costs = aot.aot_graph_costs(g.handle)
        if rule == 1:
            assert costs["walk"] == ref.walk_noclip(order)
            assert costs["positive"] == c["positive"]
        else:
            assert costs["walk"] == c["sum_deg_head"]
            assert costs["merge"] == c["sum_cf"]
            assert costs["positive"] == ref.m
        ex = g.export()
        oi, ow = ref.work_rule(rule, order)
        assert np.array_equal(ex["items"].cpu().numpy().astype(np.uint32), oi)
        assert np.array_equal(ex["walk"].cpu().numpy().astype(np.uint64), ow)


@pytest.mark.parametrize("case", ["rmat12", "rmat15", "chunglu", "path", "star", "k30", "isolated"])
def test_degeneracy_order(case):
    """eta = the degeneracy order of kClist (Sec. 2.3), peeled on the GPU:
    perm, rank and the out-CSR equal the oracle's, counts / per-vertex counts
    / list too, and with the tail rule W is kClist's sum of deg+(v)."""
    import paper_2006_11494_gb300 as aot
    if case == "rmat12":
        n, s, d = gg.rmat_cfg(12, 3)
    elif case == "rmat15":
        n, s, d = gg.rmat_cfg(15, 6)
    elif case == "chunglu":
        n = 5000
        s, d = gg.chunglu(n, 2.1, 16.0, seed=17)
    elif case == "path":
        n = 1001
        s, d = np.arange(n - 1, dtype=np.int32), np.arange(1, n, dtype=np.int32)
    elif case == "star":
        n, s, d = gg.star(300)
    elif case == "k30":
        n, s, d = gg.complete(30)
    else:
        n, s, d = 50, np.array([3, 4, 5], np.int32), np.array([4, 5, 3], np.int32)
    order = oracle.ORDER_DEGEN
    g, ref = check_full(n, s, d, flags=aot.ETA_DEGENERACY, order=order)
    rank, perm, off, adj = ref.orient(order)
    ex = g.export()
    assert np.array_equal(ex["perm"].cpu().numpy(), perm)
    assert np.array_equal(ex["rank"].cpu().numpy(), rank)
    assert np.array_equal(ex["out_off"].cpu().numpy().astype(np.int64), off)
    assert np.array_equal(ex["out_adj"].cpu().numpy(), adj)
    assert g.info["W"] == ref.costs(order)["walk"]
    gt = gpu_graph(n, s, d, aot.ETA_DEGENERACY | aot.FLAG_TAIL_PIVOT)
    assert aot.aot_graph_costs(gt.handle)["walk"] == ref.costs(order)["sum_deg_head"]
    assert gt.count() == ref.count()


def test_degeneracy_rejects_two_orders():
    import paper_2006_11494_gb300 as aot
    with pytest.raises(aot.AotError) as e:
        aot.aot_orient_workspace_size(10, 5, aot.ETA_DEGENERACY | aot.ETA_DEG_ASC)
    assert e.value.status == aot.ERR_INVALID_ARG


@pytest.mark.parametrize("tuning", [None, dict(warp_max_outdeg=8, cta_max_outdeg=64)])
def test_random_local_order(tuning):
    """AOT-randomOrder (Sec. 4.2): out-lists in a fixed pseudo-random order,
    negative items walk whole lists, hubs on the global bitmaps; counts and
    per-vertex counts equal the oracle's, W equals the oracle's W without the
    clip, the lists hold the same heads in another order, and the calls that
    need sorted lists refuse."""
    import torch
    import paper_2006_11494_gb300 as aot
    n, s, d = gg.rmat_cfg(13, 12)
    ref = oracle.Graph(n, s, d)
    T_ref, t_ref = ref.count_per_vertex()
    g = gpu_graph(n, s, d, aot.FLAG_LOCAL_RANDOM)
    if tuning:
        g.set_tuning(**tuning)
    assert g.count() == T_ref
    T, t = g.count_per_vertex()
    assert T == T_ref and np.array_equal(u64(t), t_ref)
    assert g.count(aot.ROUTE_PROBE) == T_ref
    assert aot.aot_graph_costs(g.handle)["walk"] == ref.walk_noclip()
    rank, perm, off, adj = ref.orient()
    ex = g.export()
    gadj = ex["out_adj"].cpu().numpy().astype(np.int64)
    assert np.array_equal(ex["out_off"].cpu().numpy().astype(np.int64), off)
    unsorted = 0
    for u in range(n):
        a, b = off[u], off[u + 1]
        assert np.array_equal(np.sort(gadj[a:b]), adj[a:b])
        unsorted += int(not np.array_equal(gadj[a:b], adj[a:b]))
    assert unsorted > n // 20
    for route in (aot.ROUTE_MERGE, aot.ROUTE_BSEARCH, aot.ROUTE_RANDOM):
        with pytest.raises(aot.AotError) as e:
            g.count(route)
        assert e.value.status == aot.ERR_INVALID_ARG
    out = torch.empty(30, dtype=torch.int32, device="cuda")
    with pytest.raises(aot.AotError) as e:
        aot.aot_list(g.handle, aot.ROUTE_PLAIN, 0, out, 10)
    assert e.value.status == aot.ERR_INVALID_ARG


def test_hub_wheel():
    n, s, d = gg.wheel(20000)  # hub deg+ 20000: beyond the shared-memory bins
    g, ref = check_full(n, s, d)
    assert g.info["max_outdeg"] == 20000


def test_wheel_more_segments_than_shared_bounds():
    """Wheel with a 600,000-vertex rim and 1024-rank segments: the hub's range
    spans ~586 segments, more than the shared-memory bound table holds, so the
    kernel searches each segment end.  Closed form as below."""
    rim = 600_000
    n, s, d = gg.wheel(rim)
    g = gpu_graph(n, s, d)
    g.set_tuning(seg_bits=1024)
    assert g.count() == rim
    T, t = g.count_per_vertex()
    t = u64(t)
    assert T == rim and t[0] == rim and np.all(t[1:] == 2)


@pytest.mark.parametrize("hub_mode", [0, 1])
def test_wheel_multi_segment_closed_form(hub_mode):
    """Wheel with a 3,000,000-vertex rim: the hub's out-list spans two
    1.5M-rank bitmap segments.  Closed form: T = rim, t(hub) = rim, t(rim) = 2."""
    rim = 3_000_000
    n, s, d = gg.wheel(rim)
    g = gpu_graph(n, s, d)
    g.set_tuning(hub_mode=hub_mode)
    assert g.count() == rim
    T, t = g.count_per_vertex()
    t = u64(t)
    assert T == rim and t[0] == rim and np.all(t[1:] == 2)
    lst = g.list(chunk=1 << 20).cpu().numpy()
    assert lst.shape == (rim, 3) and np.all(lst[:, 0] == 0)
    # canonical order: hub first, then rim pairs by eta (ties by id)
    assert np.all(np.diff(lst[:, 1]) >= 0)


def test_complete_dense():
    n, s, d = gg.complete(300)
    check_full(n, s, d)


# ------------------------------------------------------------- edge cases
def test_empty_and_degenerate():
    import paper_2006_11494_gb300 as aot
    e = np.zeros(0, np.int32)
    for n in (0, 1, 5):
        g = gpu_graph(n, e, e)
        assert g.m == 0 and g.count() == 0
        T, t = g.count_per_vertex()
        assert T == 0 and not u64(t).any()
        assert g.list().shape == (0, 3)
    # loops only
    g = gpu_graph(4, np.array([1, 2, 2], np.int32), np.array([1, 2, 2], np.int32))
    assert g.m == 0 and g.count() == 0
    # single edge, single triangle with duplicates, reversals and loops
    g = gpu_graph(3, np.array([0], np.int32), np.array([2], np.int32))
    assert g.m == 1 and g.count() == 0
    s = np.array([0, 1, 2, 1, 0, 2, 2], np.int32)
    d = np.array([1, 2, 0, 0, 2, 1, 2], np.int32)
    check_full(3, s, d)


def test_duplicates_reversals_loops_invariance():
    n, s, d = gg.rmat_cfg(11, 3)
    g0, ref = check_full(n, s, d)
    rng = np.random.default_rng(0)
    loops = rng.integers(0, n, 500).astype(np.int32)
    s2 = np.concatenate([d, s, loops, s[:1000]])
    d2 = np.concatenate([s, d, loops, d[:1000]])
    idx = rng.permutation(s2.size)
    g1, _ = check_full(n, s2[idx], d2[idx])
    assert g1.m == g0.m and g1.info["W"] == g0.info["W"]


def test_invalid_ids_are_rejected():
    import paper_2006_11494_gb300 as aot
    for bad in ([0, 5], [-1, 2], [2, 2147483647]):
        s = np.array([0, 1, bad[0]], np.int32)
        d = np.array([1, 2, bad[1]], np.int32)
        with pytest.raises(aot.AotError) as e:
            gpu_graph(5, s, d)
        assert e.value.status == aot.ERR_VERTEX_RANGE
    # the context stays usable
    n, s, d = gg.complete(5)
    assert gpu_graph(n, s, d).count() == 10


def test_relabel_invariance():
    n, s, d = gg.rmat_cfg(12, 9)
    g0 = gpu_graph(n, s, d)
    perm = np.random.default_rng(3).permutation(n).astype(np.int32)
    g1 = gpu_graph(n, perm[s], perm[d])
    assert g0.count() == g1.count()
    _, t0 = g0.count_per_vertex()
    _, t1 = g1.count_per_vertex()
    t0, t1 = u64(t0), u64(t1)
    assert np.array_equal(t1[perm], t0)


# ------------------------------------------------------------ listing chunks
@pytest.mark.parametrize("cap", [1, 3, 1000, 4096])
def test_chunked_listing(cap):
    import torch
    import paper_2006_11494_gb300 as aot
    n, s, d = gg.rmat_cfg(8 if cap < 10 else 10, 4)
    ref = oracle.Graph(n, s, d).list_canonical()
    g = gpu_graph(n, s, d)
    out = torch.empty(3 * cap, dtype=torch.int32, device="cuda")
    parts, cursor = [], 0
    while True:
        k, nxt = aot.aot_list(g.handle, aot.ROUTE_PLAIN, cursor, out, cap)
        assert nxt == cursor + k
        parts.append(out[: 3 * k].cpu().numpy().reshape(-1, 3))
        cursor = nxt
        if k < cap:
            break
    got = np.concatenate(parts)
    assert np.array_equal(got, ref)
    # resume from an arbitrary cursor
    mid = len(ref) // 3
    k, nxt = aot.aot_list(g.handle, aot.ROUTE_PLAIN, mid, out, cap)
    assert np.array_equal(out[: 3 * k].cpu().numpy().reshape(-1, 3), ref[mid:mid + k])
    k, nxt = aot.aot_list(g.handle, aot.ROUTE_PLAIN, len(ref), out, cap)
    assert k == 0 and nxt == len(ref)
    with pytest.raises(aot.AotError):
        aot.aot_list(g.handle, aot.ROUTE_PLAIN, len(ref) + 1, out, cap)


def test_no_list_workspace():
    import torch
    import paper_2006_11494_gb300 as aot
    n, s, d = gg.rmat_cfg(9, 4)
    g = gpu_graph(n, s, d, aot.FLAG_NO_LIST)
    assert g.count() == oracle.Graph(n, s, d).count()
    out = torch.empty(30, dtype=torch.int32, device="cuda")
    with pytest.raises(aot.AotError) as e:
        aot.aot_list(g.handle, aot.ROUTE_PLAIN, 0, out, 10)
    assert e.value.status == aot.ERR_WORKSPACE


def test_side_stream():
    import torch
    n, s, d = gg.rmat_cfg(11, 8)
    T_ref = oracle.Graph(n, s, d).count()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        src, dst = to_dev(s, d)
        import paper_2006_11494_gb300 as aot
        g = aot.OrientedGraph(src, dst, n, 0, st)
        assert g.count(stream=st) == T_ref


def test_second_device_after_the_first():
    """Kernels that need more than 48 KB of dynamic shared memory get their
    limit raised on every device they run on: orient and count on cuda:1
    after cuda:0 (skipped on a one-GPU machine)."""
    import torch
    if torch.cuda.device_count() < 2:
        pytest.skip("needs a second GPU")
    import paper_2006_11494_gb300 as aot
    n, s, d = gg.rmat_cfg(14, 3)
    ref = oracle.Graph(n, s, d)
    T_ref, t_ref = ref.count_per_vertex()
    for dev in ("cuda:0", "cuda:1"):
        with torch.cuda.device(dev):
            src = torch.from_numpy(s).to(dev)
            dst = torch.from_numpy(d).to(dev)
            g = aot.OrientedGraph(src, dst, n)
            assert g.count() == T_ref
            T, t = g.count_per_vertex()
            assert T == T_ref and np.array_equal(u64(t), t_ref)
            g.close()
