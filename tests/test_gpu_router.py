"""GPU parity of the learned router against oracle/mlp.py: tensor-core
inference, training gradients, Adam steps, features; timing capture; and the
learned route's output invariance (bit-exact counts, per-vertex counts, lists).

Tolerances (floating point): both sides round inputs, parameters and hidden
activations to bfloat16 at the same points; they differ only in the fp32 vs
fp64 accumulation order, which can move a pre-activation across a bfloat16
rounding boundary (one ulp = 2^-8 relative).  Outputs of magnitude ~1 then
differ by ~1e-3; we allow atol 2e-2 / rtol 2e-2 per element and require a
mean absolute error below 2e-3."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from oracle import mlp
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


def rand_model(seed, scale=0.4, margin=0.0):
    from paper_2006_11494_gb300 import router
    rng = np.random.default_rng(seed)
    theta = rng.normal(0, scale, mlp.NUM_PARAMS)
    in_mean = rng.normal(0, 1, 8)
    in_std = rng.uniform(0.5, 2.0, 8)
    out_mean = rng.normal(0, 1, 3)
    out_std = rng.uniform(0.5, 2.0, 3)
    buf = router.pack(theta, in_mean, in_std, out_mean, out_std, margin)
    p, im, isd, om, osd, mg = router.unpack(buf)
    return buf, mlp.unflatten(p), im.astype(np.float64), isd.astype(np.float64)


def close(got, want, atol=2e-2, rtol=2e-2, mean_tol=2e-3):
    got, want = np.asarray(got, np.float64), np.asarray(want, np.float64)
    assert got.shape == want.shape
    err = np.abs(got - want)
    assert np.all(err <= atol + rtol * np.abs(want)), float(err.max())
    assert err.mean() <= mean_tol * max(1.0, float(np.abs(want).mean())), float(err.mean())


@pytest.mark.parametrize("n", [1, 16, 37, 1037, 20000])
def test_forward_matches_oracle(aot, n):
    import torch
    buf, params, im, isd = rand_model(1)
    rng = np.random.default_rng(n)
    x = rng.normal(0, 2, (n, 8)).astype(np.float32)
    y = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    aot.aot_mlp_forward(buf, torch.from_numpy(x).cuda(), y)
    xs = (x.astype(np.float64) - im) / isd
    want, _ = mlp.forward(params, xs, exact=False)
    close(y.cpu().numpy(), want)


def test_gradient_and_loss_match_oracle(aot):
    import torch
    buf, params, im, isd = rand_model(2)
    rng = np.random.default_rng(5)
    B = 300
    x = rng.normal(0, 2, (B, 8)).astype(np.float32)
    t = rng.normal(0, 1, (B, 3)).astype(np.float32)
    ws = torch.empty(aot.aot_mlp_train_workspace_size(B), dtype=torch.uint8, device="cuda")
    grad = torch.empty(mlp.NUM_PARAMS, dtype=torch.float32, device="cuda")
    loss = aot.aot_mlp_train_step(buf, None, None, None, 1, 0.0, torch.from_numpy(x).cuda(),
                                  torch.from_numpy(t).cuda(), ws, grad_out=grad)
    xs = (x.astype(np.float64) - im) / isd
    want_loss = mlp.loss(params, xs, t.astype(np.float64))
    assert abs(loss - want_loss) <= 2e-2 * max(1.0, want_loss)
    want = mlp.flatten(mlp.backward(params, xs, t.astype(np.float64)))
    got = grad.cpu().numpy().astype(np.float64)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 2e-2 * scale
    assert np.abs(got - want).mean() <= 2e-3 * scale


def test_adam_steps_match_oracle(aot):
    import torch
    from paper_2006_11494_gb300 import router
    buf, params, im, isd = rand_model(3, scale=0.2)
    rng = np.random.default_rng(9)
    B = 128
    x = rng.normal(0, 1, (B, 8)).astype(np.float32)
    t = rng.normal(0, 1, (B, 3)).astype(np.float32)
    theta = mlp.flatten(params)
    master = torch.from_numpy(theta.astype(np.float32)).cuda()
    m1 = torch.zeros_like(master)
    m2 = torch.zeros_like(master)
    ws = torch.empty(aot.aot_mlp_train_workspace_size(B), dtype=torch.uint8, device="cuda")
    xs = (x.astype(np.float64) - im) / isd
    ref, rm, rv = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for step in (1, 2, 3):
        aot.aot_mlp_train_step(buf, master, m1, m2, step, 1e-2, torch.from_numpy(x).cuda(),
                               torch.from_numpy(t).cuda(), ws)
        g = mlp.flatten(mlp.backward(mlp.unflatten(mlp.bf16(ref)), xs, t.astype(np.float64)))
        ref, rm, rv = mlp.adam(ref, g, rm, rv, step, 1e-2)
    got = master.cpu().numpy().astype(np.float64)
    # Adam moves each weight by ~lr per step; allow a tenth of that per weight
    assert np.abs(got - ref).max() <= 3e-3
    # the model now holds the bf16 rounding of the master copy
    p, *_ = router.unpack(buf)
    assert np.array_equal(p, mlp.bf16(got))


def test_features_match_oracle(aot):
    import torch
    n, s, d = gg.rmat_cfg(11, 31)
    ref = oracle.Graph(n, s, d)
    rank, perm, off, adj = ref.orient()
    deg_rank = ref.degrees()[perm]
    want = mlp.features(off, adj, deg_rank)
    g = gpu_graph(n, s, d)
    f = torch.empty((g.m, 8), dtype=torch.float32, device="cuda")
    aot.aot_graph_features(g.handle, f)
    got = f.cpu().numpy().astype(np.float64)
    assert np.allclose(got, want, rtol=1e-6, atol=1e-6)


def test_record_costs(aot):
    import torch
    n, s, d = gg.rmat_cfg(12, 32)
    g = gpu_graph(n, s, d)
    c = torch.zeros(g.m, dtype=torch.int32, device="cuda")
    aot.aot_graph_record_costs(g.handle, 0, c)
    assert bool((c != 0).all())
    for v in (1, 2):
        c.zero_()
        aot.aot_graph_record_costs(g.handle, v, c, 4)
        frac = float((c != 0).float().mean())
        assert 0.03 < frac < 0.10, frac  # about 1/16 of the items
        c.zero_()
        aot.aot_graph_record_costs(g.handle, v, c)
        assert bool((c != 0).all())
    # counting still works after timing runs
    assert g.count() == oracle.Graph(n, s, d).count()


@pytest.mark.parametrize("margin", [-100.0, 0.0, 100.0])
def test_learned_route_is_invisible_in_the_output(aot, margin):
    n, s, d = gg.rmat_cfg(12, 33)
    ref = oracle.Graph(n, s, d)
    T_ref, t_ref = ref.count_per_vertex()
    lst_ref = ref.list_canonical()
    buf, *_ = rand_model(4, margin=margin)
    g = gpu_graph(n, s, d)
    with pytest.raises(aot.AotError) as e:
        g.count(aot.ROUTE_LEARNED)
    assert e.value.status == aot.ERR_NOT_READY
    aot.aot_graph_set_router(g.handle, buf)
    assert g.count(aot.ROUTE_LEARNED) == T_ref
    T, t = g.count_per_vertex(aot.ROUTE_LEARNED)
    assert T == T_ref and np.array_equal(u64(t), t_ref)
    assert np.array_equal(g.list(aot.ROUTE_LEARNED, chunk=50000).cpu().numpy(), lst_ref)


@pytest.mark.slow
def test_learned_vs_plain_on_the_held_out_graph(aot):
    """The committed router on the graph held out of its training (R-MAT s22,
    seed 1019): the learned route at the committed margin and at margin 0 (the
    network's own choice, which reroutes items) gives the plain route's exact
    count and per-vertex counts; the measured speed-up is printed."""
    import torch
    from paper_2006_11494_gb300 import router
    model = router.load()
    assert model is not None
    n, s, d = gg.rmat_cfg(22, 1019)
    g = gpu_graph(n, s, d, aot.FLAG_NO_LIST)
    T0, t0 = g.count_per_vertex()
    t0 = u64(t0)

    def timed(route):
        best = 1e30
        for _ in range(3):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record()
            T = g.count(route)
            b.record()
            torch.cuda.synchronize()
            best = min(best, a.elapsed_time(b))
        return T, best

    T_plain, ms_plain = timed(aot.ROUTE_PLAIN)
    for margin in (None, 0.0):
        buf = model if margin is None else router.with_margin(model, margin)
        aot.aot_graph_set_router(g.handle, buf)
        T, ms = timed(aot.ROUTE_LEARNED)
        Tv, tv = g.count_per_vertex(aot.ROUTE_LEARNED)
        assert T == T_plain == Tv == T0
        assert np.array_equal(u64(tv), t0)
        print("held-out R-MAT s22: plain %.2f ms, learned (margin %s) %.2f ms, speed-up %.3f"
              % (ms_plain, "committed" if margin is None else margin, ms, ms_plain / ms))
    aot.aot_graph_set_router(g.handle, None)
