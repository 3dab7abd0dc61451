"""Train the learned router on the GPU with the library's own kernels.

1. Training graphs: R-MAT (.57,.19,.19,.05), edge factor 16, scales 18-22,
   seeds 1000-1019 (disjoint from every benchmark and test seed).
2. Labels: per-item cycles recorded by the intersection kernels themselves
   (aot_graph_record_costs) for the probe, merge and binary-search variants;
   the slow variants are timed on a hashed sample of the items.
3. Features: aot_graph_features (eight per oriented edge).
4. Network: 8 -> 64 -> 64 -> 3, regression of the standardised log1p cycles,
   trained with aot_mlp_train_step (bf16 forward/backward kernels, fp32
   accumulation, Adam on an fp32 master copy).
5. Margin: the plain rule judges the network.  On a held-out graph the count
   is timed with the plain route and with the learned route at several
   margins; the fastest margin is kept (a margin so large that nothing moves
   is the plain rule itself).

    python -m paper_2006_11494_gb300.train_router [--out FILE] [--quick]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import graphgen  # noqa: E402
import paper_2006_11494_gb300 as aot  # noqa: E402
from paper_2006_11494_gb300 import router  # noqa: E402


def he_init(seed):
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0, math.sqrt(2 / 8), (64, 8)), np.zeros(64),
             rng.normal(0, math.sqrt(2 / 64), (64, 64)), np.zeros(64),
             rng.normal(0, math.sqrt(1 / 64), (3, 64)), np.zeros(3)]
    return np.concatenate([p.ravel() for p in parts])


def collect(scale, seed, per_graph, sample_log2, rng):
    import torch
    n, s, d = graphgen.rmat_cfg(scale, seed)
    g = aot.OrientedGraph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n, aot.FLAG_NO_LIST)
    m = g.m
    feat = torch.empty((m, 8), dtype=torch.float32, device="cuda")
    aot.aot_graph_features(g.handle, feat)
    cyc = torch.zeros((3, m), dtype=torch.int32, device="cuda")
    aot.aot_graph_record_costs(g.handle, 0, cyc[0])
    aot.aot_graph_record_costs(g.handle, 1, cyc[1], sample_log2)
    aot.aot_graph_record_costs(g.handle, 2, cyc[2], sample_log2)
    ok = ((cyc != 0).all(dim=0)).nonzero().flatten()
    if ok.numel() > per_graph:
        ok = ok[torch.from_numpy(rng.choice(ok.numel(), per_graph, replace=False)).cuda()]
    x = feat[ok].cpu()
    c = cyc[:, ok].T.contiguous().view(torch.int32).cpu().numpy().astype(np.uint32)
    g.close()
    return x.numpy(), c


def time_count(g, route, reps=3):
    import torch
    best = 1e30
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record()
        g.count(route)
        b.record()
        torch.cuda.synchronize()
        best = min(best, a.elapsed_time(b))
    return best


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=router.DEFAULT_MODEL_PATH)
    ap.add_argument("--quick", action="store_true", help="smaller graphs and fewer steps")
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=4096)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--per-graph", type=int, default=60000)
    a = ap.parse_args()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(7)
    scales = [14, 15, 16] if a.quick else [18, 19, 20, 21, 22]
    seeds = list(range(1000, 1004 if a.quick else 1020))
    t0 = time.time()
    X, C = [], []
    for i, seed in enumerate(seeds[:-1]):
        sc = scales[i % len(scales)]
        x, c = collect(sc, seed, a.per_graph, 0 if sc <= 18 else 4, rng)
        X.append(x)
        C.append(c)
        print("collected scale %d seed %d: %d items (%.1fs)" % (sc, seed, len(x), time.time() - t0), flush=True)
    X = np.concatenate(X).astype(np.float32)
    Call = np.concatenate(C).astype(np.float64)
    # upper bound of any per-item route on these items: every item in its
    # cheapest variant, by its own recorded cycles
    bound = float(Call[:, 0].sum() / Call.min(axis=1).sum())
    print("perfect per-item routing on the sampled items: %.3fx the probe route" % bound, flush=True)
    Y = np.log1p(Call).astype(np.float32)
    in_mean, in_std = X.mean(0), X.std(0) + 1e-3
    out_mean, out_std = Y.mean(0), Y.std(0) + 1e-3
    T = ((Y - out_mean) / out_std).astype(np.float32)
    perm = rng.permutation(len(X))
    nval = max(1, len(X) // 20)
    val, tr = perm[:nval], perm[nval:]
    xd = torch.from_numpy(X).cuda()
    td = torch.from_numpy(T).cuda()
    theta = he_init(11)
    model = router.pack(theta, in_mean, in_std, out_mean, out_std, 0.0)
    master = torch.from_numpy(theta.astype(np.float32)).cuda()
    m1 = torch.zeros_like(master)
    m2 = torch.zeros_like(master)
    ws = torch.empty(aot.aot_mlp_train_workspace_size(a.batch), dtype=torch.uint8, device="cuda")
    wsv = torch.empty(aot.aot_mlp_train_workspace_size(len(val)), dtype=torch.uint8, device="cuda")
    trd = torch.from_numpy(tr).cuda()
    steps = 400 if a.quick else a.steps
    for step in range(1, steps + 1):
        bi = trd[torch.randint(0, len(tr), (a.batch,), device="cuda")]
        lr = a.lr * (0.5 * (1 + math.cos(math.pi * step / steps)))
        want = step % 200 == 0 or step == steps
        loss = aot.aot_mlp_train_step(model, master, m1, m2, step, lr, xd[bi].contiguous(),
                                      td[bi].contiguous(), ws, want_loss=want)
        if want:
            vi = torch.from_numpy(val).cuda()
            vloss = aot.aot_mlp_train_step(model, None, None, None, 1, 0.0, xd[vi].contiguous(),
                                           td[vi].contiguous(), wsv)
            print("step %d train loss %.4f val loss %.4f" % (step, loss, vloss), flush=True)
    # margin chosen by the plain rule on a held-out graph
    sc_val = 20 if a.quick else 22
    n, s, d = graphgen.rmat_cfg(sc_val, seeds[-1])
    g = aot.OrientedGraph(torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n, aot.FLAG_NO_LIST)
    t_plain = time_count(g, aot.ROUTE_PLAIN)
    T_plain = g.count(aot.ROUTE_PLAIN)
    results = {"plain_ms": t_plain}
    best_margin, best_ms = 1e9, t_plain
    for margin in (0.0, 0.1, 0.25, 0.5, 1.0, 2.0):
        mb = router.with_margin(model, margin)
        aot.aot_graph_set_router(g.handle, mb)
        assert g.count(aot.ROUTE_LEARNED) == T_plain
        ms = time_count(g, aot.ROUTE_LEARNED)
        results["margin_%.2f_ms" % margin] = ms
        print("validation scale %d: plain %.2f ms, learned margin %.2f: %.2f ms" % (sc_val, t_plain, margin, ms), flush=True)
        if ms < best_ms:
            best_margin, best_ms = margin, ms
    params, im, isd, om, osd, _ = router.unpack(model)
    meta = {"train_graphs": ["rmat s%d seed %d" % (scales[i % len(scales)], sd) for i, sd in enumerate(seeds[:-1])],
            "validation_graph": "rmat s%d seed %d" % (sc_val, seeds[-1]), "steps": steps,
            "batch": a.batch, "items": int(len(X)), "timings_ms": results,
            "chosen_margin": best_margin, "speedup_on_validation": t_plain / best_ms,
            "perfect_item_routing_bound": bound}
    router.save(a.out, params, im, isd, om, osd, best_margin, meta)
    print(json.dumps(meta), flush=True)


if __name__ == "__main__":
    main()
