"""Benchmark of the AOT hot path on GB300.

One step = the whole hot path over one synthetic graph resident in HBM:
orientation (cleanup, eta, oriented CSR, work items, bins) followed by the
per-vertex triangle count (walk + probe of Algorithm 3, every pivot's index
built once).  Workload: R-MAT scale 24, edge factor 16, (a,b,c,d) =
(.57,.19,.19,.05), ids permuted, seed 3 (synthetic stand-in for the paper's
real graphs).  Metric: oriented edges per second (m / step time); the JSON
line also carries triangles per second, the count-phase time, and the
roofline of the dominant kernel measured with CUDA events inside the timed
region.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the slow reference program of this
project) on a bounded prefix sample of the same edge stream.
Under torchrun (N > 1) every rank runs an independent replica of the
workload (the graph is not sharded: replicas only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "oriented edges/s & triangles/s at R-MAT s24, learned vs plain; HBM roofline frac"
UNIT = "oriented edges/s"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
# The oracle (cleanup + parallel per-vertex count on every host core) runs on
# the first 2^CPU_SAMPLE_LOG2 pairs of the benchmark's edge stream: the full
# 2^28-pair graph takes minutes of host time, this prefix tens of seconds.
CPU_SAMPLE_LOG2 = 27

# DRAM traffic per launch of the dominant kernel on the default workload, from
# one ncu capture of this command's timed launch (dram__bytes_read.sum +
# dram__bytes_write.sum, a one-pass metric set, taken right after the same
# command exited 0 without ncu).  It stands only for the kernel sources and
# tuning it was taken with: any change reports null.
MEASURED_TRAFFIC = {
    ("k_seg_pivots/vertex", 24, 3): {
        "bytes": 680453169408 + 6267329280,
        "sources": {
            "paper_2006_11494_gb300/csrc/aot_count.cu":
                "8bf5a28bf980dff9211a10d7d8ceea11878ba83245b14397e25eaba2064bea3e",
            "paper_2006_11494_gb300/csrc/aot_kparams.cuh":
                "eaaa7f4c852be23ebc83425f0e7c2203abb4a356c5c241c476eef2b73021acc4",
            "paper_2006_11494_gb300/csrc/aot_internal.cuh":
                "8a55c942dd024949a61507c99f83d3924131c359f3441faaf52892c70b77d396",
        },
        "tuning": {"warp_max_outdeg": 64, "cta_max_outdeg": 512, "cta_threads": 32, "hub_bitmaps": 32,
                   "hub_mode": 0, "seg_bits": 1310720, "seg_long": 128, "seg_wide": 512, "tile_bits": 0,
                   "seg_tail": 128, "seg_threads": 1024, "seg_hash": 12288},
    },
}


def workload_name(scale, seed):
    """The workload both arms name in their config."""
    return ("R-MAT scale %d edge factor 16 (a,b,c,d)=(.57,.19,.19,.05) seed %d, "
            "eta = degree non-increasing" % (scale, seed))


def workload_config(scale, seed):
    """The config both arms print (identical, so that the arms compare)."""
    return {"workload": workload_name(scale, seed), "n": 1 << scale, "generated_edges": 16 << scale,
            "l2": "inputs larger than L2 (2 GB edge list, 129 MB L2)"}


def cpu_model():
    """CPU model name of this host (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def measured_traffic(kernel, scale, seed, tuning):
    """Bytes per launch from MEASURED_TRAFFIC when the sources and tuning still match, else None."""
    import hashlib
    e = MEASURED_TRAFFIC.get((kernel, scale, seed))
    if not e or tuning != e["tuning"]:
        return None
    for rel, digest in e["sources"].items():
        with open(os.path.join(ROOT, rel), "rb") as f:
            if hashlib.sha256(f.read()).hexdigest() != digest:
                return None
    return e["bytes"]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=24)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--route", default="plain", choices=["plain", "learned"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-log2", type=int, default=CPU_SAMPLE_LOG2,
                    help="log2 of the edge-stream prefix the CPU baseline and the reference arm run on")
    ap.add_argument("--cpu-threads", type=int, default=0,
                    help="host threads of the CPU baseline and the reference arm (0: all cores)")
    ap.add_argument("--no-tune", action="store_true", help="skip the autotuner (built-in tuning)")
    ap.add_argument("--tuning", default=None,
                    help="JSON object of aot_tuning fields to use instead of autotuning")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the learned-vs-plain and eta-order ablation measurements")
    return ap.parse_args()


# -------------------------------------------------------------- utilities
def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (the step time every rank reports);
    x itself when not running distributed."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(units_per_rank: float, max_ms: float, world: int) -> float:
    """Whole-job throughput of N independent replicas: the units all ranks
    processed divided by the slowest rank's time per step."""
    return world * units_per_rank / (max_ms / 1e3)


def measured_peak():
    try:
        with open(PEAKS_FILE) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", "aot_clocks_%d_%d.csv" % (os.getpid(), gpu_index))

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


_HOST_MAPS = []  # keeps the mappings behind registered host buffers alive


def pinned_host(count, np_dtype, torch):
    """A page-locked host array backed by transparent huge pages where the
    kernel offers them (an mmap aligned to the huge-page size, madvise,
    touched, then cudaHostRegister): the GPU's copies then translate a few
    huge pages instead of tens of thousands of base pages.  Falls back to
    torch's pinned allocator."""
    import mmap
    import ctypes
    import numpy as np
    nbytes = int(count) * np.dtype(np_dtype).itemsize
    try:
        hp = int(open("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size").read())
    except Exception:
        hp = 2 << 20
    try:
        size = (nbytes + hp - 1) // hp * hp
        m = mmap.mmap(-1, size + hp, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        base = ctypes.addressof(ctypes.c_char.from_buffer(m))
        off = (-base) % hp
        if hasattr(m, "madvise") and hasattr(mmap, "MADV_HUGEPAGE"):
            m.madvise(mmap.MADV_HUGEPAGE, off, size)
        arr = np.frombuffer(m, dtype=np.uint8, count=nbytes, offset=off).view(np_dtype)
        arr.fill(0)
        if torch.cuda.cudart().cudaHostRegister(arr.ctypes.data, nbytes, 0) != 0:
            raise RuntimeError("cudaHostRegister failed")
        _HOST_MAPS.append(m)
        t = torch.from_numpy(arr)
        if t.is_pinned():
            return t
    except Exception:
        pass
    return torch.empty(int(count), dtype=getattr(torch, np.dtype(np_dtype).name)).pin_memory()


# ------------------------------------------------------- algorithmic bytes
def bytes_per_kernel(info, bins, E, n):
    """Algorithmic HBM bytes of one step, per kernel family: the radix sort
    reads every key once for its histograms and moves every key (and value)
    once per pass; an intersection bin
    stages N+(p) of its pivots, reads their offsets and their items' walk
    ranges and walked vertices, and every walked adjacency entry once."""
    m, bits = info["m"], max(1, math.ceil(math.log2(max(n, 2))))
    passes_keys = math.ceil(2 * bits / 8)
    passes_eta = math.ceil(bits / 8)
    out = {}
    # radix sort: each sweep reads and writes every key (and value) once
    out["k_onesweep"] = (passes_keys * (16 * E + 16 * m) + passes_eta * 16 * n,
                         2 * passes_keys + passes_eta)
    out["k_digit_hist"] = (8 * E + 8 * m + 4 * n, 3)

    def walk_bytes(b):
        st = bins[b]
        # stage N+(p), read the pivot's offsets, the items' walk ranges and
        # walked vertices, and every walked adjacency entry once
        return 4 * st["staged"] + 16 * st["pivots"] + 12 * st["items"] + 4 * st["walk"]

    out["k_warp_pivots/vertex"] = (walk_bytes("warp"), 1)
    out["k_cta_pivots/vertex"] = (walk_bytes("cta"), 1)
    out["k_warp_pivots_ctabin/vertex"] = (walk_bytes("cta"), 1)  # the CTA bin a warp per pivot
    out["k_seg_pivots/vertex"] = (walk_bytes("hub"), 1)
    out["k_hub_walk/vertex"] = (walk_bytes("hub") - 4 * bins["hub"]["staged"], None)
    return out


# The paper's algorithms and ablations on the same graph (Sec. 2.2, 2.3, 4.2):
# (name, orientation flags, route, work counter that bounds it)
VARIANTS = [
    ("AOT, eta degree non-increasing (the benchmark)", 0, "ROUTE_PLAIN", "walk"),
    ("AOT, eta degree non-decreasing", "ETA_DEG_ASC", "ROUTE_PLAIN", "walk"),
    ("AOT, eta degeneracy", "ETA_DEGENERACY", "ROUTE_PLAIN", "walk"),
    ("AOT without the suffix clip (Algorithm 3 as printed)", "FLAG_NO_CLIP", "ROUTE_PLAIN", "walk"),
    ("AOT-randomOrder (random local order, Sec. 4.2)", "FLAG_LOCAL_RANDOM", "ROUTE_PLAIN", "walk"),
    ("kClist work: degeneracy eta, every edge from its tail, index probe (Algorithm 2)",
     "ETA_DEGENERACY|FLAG_TAIL_PIVOT", "ROUTE_PLAIN", "walk"),
    ("kClist work on eta degree non-increasing", "FLAG_TAIL_PIVOT", "ROUTE_PLAIN", "walk"),
    ("CF: degree non-decreasing eta, every edge from its tail, merge (Algorithm 1)",
     "ETA_DEG_ASC|FLAG_TAIL_PIVOT", "ROUTE_MERGE", "merge"),
]


def variants(aot, src, dst, n, ws, stream, phase_ms, T_ref):
    """Orientation time, work counter and count time of every variant; the
    triangle count must equal the benchmark's."""
    import torch
    out = []
    for name, flags, route, work in VARIANTS:
        f = aot.FLAG_NO_LIST
        if flags:
            for part in flags.split("|"):
                f |= getattr(aot, part)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        h = aot.aot_orient(src, dst, n, f, ws, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        c = aot.aot_graph_costs(h)
        r = getattr(aot, route)
        T = aot.aot_count(h, r, stream)
        ms = phase_ms(lambda: aot.aot_count(h, r, stream), 2)
        aot.aot_graph_destroy(h)
        out.append({"variant": name, "orient_ms": e0.elapsed_time(e1), "work": work,
                    "work_entries": c[work], "count_ms": ms, "same_T": T == T_ref})
    return out


def count_phase_bytes(info, n):
    """Algorithmic bytes of the whole count phase: stage N+(p) (4 S), the
    items (12 m: walk range and walked vertex), the walked entries (4 W), the
    pivot offsets (8 (n+1)) and the per-vertex output (8 n)."""
    return 4 * info["S"] + 12 * info["m"] + 4 * info["W"] + 8 * (n + 1) + 8 * n


# ------------------------------------------------------------------ ours
def run_ours(a):
    import numpy as np
    import torch
    import graphgen as gg
    import paper_2006_11494_gb300 as aot

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n = 1 << a.scale
    E = 16 << a.scale
    h_src = pinned_host(E, np.int32, torch)
    h_dst = pinned_host(E, np.int32, torch)
    gg.rmat(a.scale, 16, a.seed, out=(h_src.numpy(), h_dst.numpy()))
    src = h_src.to(dev)
    dst = h_dst.to(dev)
    ws_bytes = aot.aot_orient_workspace_size(E, n, aot.FLAG_NO_LIST)
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device=dev)
    counts = torch.empty(n, dtype=torch.int64, device=dev)
    h_counts = pinned_host(n, np.int64, torch)
    route = aot.ROUTE_PLAIN if a.route == "plain" else aot.ROUTE_LEARNED
    stream = torch.cuda.current_stream(dev)

    def step(s_src, s_dst):
        h = aot.aot_orient(s_src, s_dst, n, aot.FLAG_NO_LIST, ws, stream)
        aot.aot_count_per_vertex(h, route, counts, want_total=False, stream=stream)
        return h

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # autotune once on this workload (per-vertex mode); later graphs inherit it
    tuning, tune_ms = None, None
    if a.tuning:
        t = aot.aot_get_default_tuning()
        for k, v in json.loads(a.tuning).items():
            setattr(t, k, v)
        aot.aot_set_default_tuning(t)
        tuning = t.as_dict()
    elif not a.no_tune:
        h = aot.aot_orient(src, dst, n, aot.FLAG_NO_LIST, ws, stream)
        t, tune_ms = aot.aot_tune(h, 1, 1, stream)
        aot.aot_set_default_tuning(t)
        tuning = t.as_dict()
        aot.aot_graph_destroy(h)
    # warm-up (also the reference values of this run)
    for _ in range(max(a.warmup, 3)):
        h = step(src, dst)
        info = aot.aot_graph_info(h)
        bins = aot.aot_graph_bins(h)
        aot.aot_graph_destroy(h)
    torch.cuda.synchronize()
    T = int(counts.sum().item()) // 3

    # timed region: K steps, inputs resident in HBM (2 GB edge list > L2),
    # no per-launch events
    l0 = aot.aot_kernel_launches()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(a.steps):
            aot.aot_graph_destroy(step(src, dst))
        ev1.record(stream)
        torch.cuda.synchronize()
        barrier()
    launches = aot.aot_kernel_launches() - l0
    ms = max_over_ranks(ev0.elapsed_time(ev1) / a.steps, dev)
    # the same K steps again with a pair of CUDA events around every launch
    # (on its stream): per-kernel durations for the roofline
    aot.aot_profile_begin()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    p0.record(stream)
    for _ in range(a.steps):
        aot.aot_graph_destroy(step(src, dst))
    p1.record(stream)
    torch.cuda.synchronize()
    prof = aot.aot_profile_end()
    profiled_ms = p0.elapsed_time(p1) / a.steps

    # count phase alone, for context: plain route, learned route, count mode
    def phase_ms(fn, reps):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        c0.record(stream)
        for _ in range(reps):
            fn()
        c1.record(stream)
        torch.cuda.synchronize()
        return c0.elapsed_time(c1) / reps

    h = aot.aot_orient(src, dst, n, aot.FLAG_NO_LIST, ws, stream)
    count_ms = phase_ms(lambda: aot.aot_count_per_vertex(h, route, counts, want_total=False,
                                                         stream=stream), a.steps)
    extras = {}
    if not a.no_extras:
        from paper_2006_11494_gb300 import router as rt
        count_only_ms = phase_ms(lambda: aot.aot_count(h, aot.ROUTE_PLAIN, stream), a.steps)
        extras["count_only_ms"] = count_only_ms
        extras["count_only_hbm_frac"] = count_phase_bytes(info, n) / (count_only_ms / 1e3) / 1e9 / measured_peak()[0]
        model = rt.load()
        if model is not None:
            aot.aot_graph_set_router(h, model)
            plain = phase_ms(lambda: aot.aot_count(h, aot.ROUTE_PLAIN, stream), a.steps)
            learned = phase_ms(lambda: aot.aot_count(h, aot.ROUTE_LEARNED, stream), a.steps)
            forced = rt.with_margin(model, 0.0)  # the network's own choice, no plain-rule margin
            aot.aot_graph_set_router(h, forced)
            learned0 = phase_ms(lambda: aot.aot_count(h, aot.ROUTE_LEARNED, stream), a.steps)
            aot.aot_graph_set_router(h, None)
            extras["learned_vs_plain"] = {
                "plain_count_ms": plain, "learned_count_ms": learned,
                "speedup": plain / learned, "learned_margin0_count_ms": learned0,
                "speedup_margin0": plain / learned0,
                "note": "model trained on R-MAT s18-22 timings; the plain rule judged it on a held-out graph"}
    aot.aot_graph_destroy(h)
    if not a.no_extras:
        extras["variants"] = variants(aot, src, dst, n, ws, stream, phase_ms, T)

    # end to end: pinned host edge list in, per-vertex counts out, every step,
    # in two pipelines a user may run: each step's input copied on a copy
    # stream into one of two device buffers while the previous step computes,
    # or copy then compute.  The host-to-device copy runs at very different
    # speeds beside the bandwidth-bound count kernel from one GPU machine to the
    # next, so either can be the faster: the value is the faster one, and both
    # times are in the line.
    e2e = None
    if not a.no_e2e:
        o_ms, o_wall = e2e_loop(torch, aot, step, src, dst, h_src, h_dst, counts, h_counts, stream,
                                a.steps, True, barrier)
        s_ms, s_wall = e2e_loop(torch, aot, step, src, dst, h_src, h_dst, counts, h_counts, stream, a.steps,
                                False, barrier)
        o_ms = max_over_ranks(o_ms, dev)
        s_ms = max_over_ranks(s_ms, dev)
        overlap_wins = o_ms <= s_ms
        e_ms = o_ms if overlap_wins else s_ms
        e2e = {"value": replica_value(info["m"], e_ms, world), "unit": UNIT, "ms_per_step": e_ms,
               "wall_ms_per_step": o_wall if overlap_wins else s_wall,
               "h2d_bytes_per_step": 8 * E, "d2h_bytes_per_step": 8 * n,
               "copies": ("overlapped with the previous step (two input buffers, a copy stream)" if overlap_wins
                          else "serial: copy in, then orient + count, then copy out"),
               "overlapped_ms_per_step": o_ms, "serial_ms_per_step": s_ms}

    if rank != 0:
        return
    # roofline of the dominant kernel
    peak, peak_kind = measured_peak()
    bpk = bytes_per_kernel(info, bins, E, n)
    dom = max(prof.items(), key=lambda kv: kv[1][1]) if prof else None
    roof = None
    if dom:
        name, (nl, tot_ms) = dom
        per_launch_ms = tot_ms / nl
        b = bpk.get(name)
        if b:
            total_bytes, lpstep = b
            lps = nl / a.steps
            per_launch_bytes = total_bytes / lps
            achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
            traffic = measured_traffic(name, a.scale, a.seed, tuning)
            roof = {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak,
                    "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                    "traffic": traffic, "launch_ms": per_launch_ms, "alg_bytes_per_launch": per_launch_bytes,
                    "traffic_over_alg": traffic / per_launch_bytes if traffic else None}
        else:
            roof = {"bound": "hbm", "kernel": name, "achieved": None, "peak": peak, "unit": "GB/s",
                    "frac": None, "traffic": None}
    total_prof = sum(v[1] for v in prof.values()) or 1.0
    kernels = {k: {"launches": v[0], "ms": round(v[1], 4), "share": round(v[1] / total_prof, 4)}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    cpu = None
    if not a.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(a.scale, a.seed, a.cpu_sample_log2, a.cpu_threads, h_src.numpy(),
                           h_dst.numpy())

    value = replica_value(info["m"], ms, world)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
        "warmup": a.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(a.scale, a.seed),
        "parallelism": "replicas" if world > 1 else "1 GPU",
        "step": "aot_orient + aot_count_per_vertex (%s route)" % a.route,
        "graph": {"m": info["m"], "W": info["W"], "S": info["S"], "max_outdeg": info["max_outdeg"],
                  "triangles": T},
        "profiled_ms_per_step": profiled_ms,
        "triangles_per_s": world * T / (ms / 1e3),
        "count_phase": {"ms": count_ms, "oriented_edges_per_s": info["m"] / (count_ms / 1e3),
                        "triangles_per_s": T / (count_ms / 1e3), "probes_per_s": info["W"] / (count_ms / 1e3),
                        "alg_bytes": count_phase_bytes(info, n),
                        "hbm_frac": count_phase_bytes(info, n) / (count_ms / 1e3) / 1e9 / measured_peak()[0]},
        "tuning": {"autotuned": tuning is not None and not a.tuning, "values": tuning, "tune_best_ms": tune_ms},
        "extras": extras,
        "bins": bins,
        "roofline": roof,
        "kernels": kernels,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


def e2e_loop(torch, aot, step, src, dst, h_src, h_dst, counts, h_counts, stream, steps, overlap, barrier):
    """K steps from pinned host memory: copy the edge list in (copy stream),
    orient + count, read the per-vertex counts back; with overlap, step i+1's
    input is copied into the other buffer while step i computes.  Returns the
    event time on the compute stream and the wall time per step (ms)."""
    cs = torch.cuda.Stream(src.device)
    bufs = [(torch.empty_like(src), torch.empty_like(dst)) for _ in range(2 if overlap else 1)]
    ready = [torch.cuda.Event() for _ in bufs]
    free = [torch.cuda.Event() for _ in bufs]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def load(i):
        b = i % len(bufs)
        cs.wait_event(e0 if i < len(bufs) else free[b])
        with torch.cuda.stream(cs):
            bufs[b][0].copy_(h_src, non_blocking=True)
            bufs[b][1].copy_(h_dst, non_blocking=True)
        ready[b].record(cs)

    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e0.record(stream)
    if overlap:
        load(0)
    for i in range(steps):
        b = i % len(bufs)
        if not overlap:
            load(i)
        elif i + 1 < steps:
            load(i + 1)
        stream.wait_event(ready[b])
        aot.aot_graph_destroy(step(*bufs[b]))
        free[b].record(stream)
        h_counts.copy_(counts, non_blocking=True)
        stream.synchronize()
    e1.record(stream)
    torch.cuda.synchronize()
    wall = (time.perf_counter() - t0) * 1e3 / steps
    return e0.elapsed_time(e1) / steps, wall


# ------------------------------------------------------------ CPU oracle
def oracle_step(n, src, dst, threads):
    """One step of the oracle as it stands: cleanup (og_new_par) and the
    parallel per-vertex count (og_count_par) on `threads` host threads."""
    import oracle
    g = oracle.Graph(n, src, dst, threads=threads)
    T, _ = g.count_per_vertex_par(threads)
    return g.m, T


def sample_text(scale, log2_sample, m, T, cores):
    return ("first 2^%d of the %d generated pairs of the same R-MAT stream (m=%d oriented edges, "
            "T=%d; sparser in triangles than the full graph): cleanup + per-vertex count, "
            "%d host threads (%s)" % (log2_sample, 16 << scale, m, T, cores, cpu_model()))


def cpu_baseline(scale, seed, log2_sample, threads, src_np, dst_np):
    """The oracle, as it stands, on a prefix of the same edge stream, on every
    host core."""
    import oracle
    n = 1 << scale
    E = 1 << log2_sample
    cores = oracle.host_threads(threads)
    t0 = time.perf_counter()
    m, T = oracle_step(n, src_np[:E], dst_np[:E], cores)
    dt = time.perf_counter() - t0
    return {"value": m / dt, "unit": UNIT, "cores": cores, "kind": "oracle", "seconds": dt,
            "sample": sample_text(scale, log2_sample, m, T, cores)}


def run_reference(a):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import graphgen as gg
    import oracle
    log2_sample = a.cpu_sample_log2
    E = 1 << log2_sample
    n = 1 << a.scale
    cores = oracle.host_threads(a.cpu_threads)
    # the first E pairs of the same stream (pairs are drawn independently)
    src, dst = gg.rmat(a.scale, 16, a.seed, num_edges=E)
    for _ in range(a.warmup):
        oracle_step(n, src, dst, cores)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        m, T = oracle_step(n, src, dst, cores)
    dt = (time.perf_counter() - t0) / a.steps
    v = m / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config(a.scale, a.seed),
        "parallelism": "%d host threads" % cores,
        "step": "oracle cleanup + per-vertex count of a bounded sample of the workload",
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample_text(a.scale, log2_sample, m, T, cores)},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
