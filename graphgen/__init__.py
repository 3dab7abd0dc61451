"""Seeded synthetic graph inputs shared by the oracle tests, the CUDA path tests
and the benchmark.

This module holds no part of the triangle method: it only produces undirected
int32 edge lists (which may contain self-loops and duplicate or reversed
pairs).  The heavy generators live in ``graphgen.c`` (compiled with gcc on
first use or by :func:`build`); the closed-form graphs below are tiny numpy
constructions used as pins.

Workload recipes (the synthetic stand-ins for the paper's real graphs, whose
shape is described in its Table 2: average degree 4-53, maximum degree
10^3.5-10^6.5):

* ``er_16k``     Erdos-Renyi, n = 16384, 262144 uniform pairs, seed 1
* ``rmat(s)``    R-MAT scale s, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
                 ids relabelled by a seeded permutation
* ``chunglu``    Chung-Lu, weights ~ (i+1)^(-1/(gamma-1)), mean degree d
* ``batch``      4096 Chung-Lu graphs, n log-uniform in [256, 65536], mean
                 degree uniform in [4, 64], gamma = 2.5, per-graph seeds
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "_build", "libgraphgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile libgraphgen.so (gcc, -O3, pthreads) next to the source."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O3", "-std=c11", "-fPIC", "-shared", "-pthread",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i32p = ctypes.c_void_p
        lib.gg_er.argtypes = [ctypes.c_uint32, ctypes.c_int64, ctypes.c_uint64, i32p, i32p, ctypes.c_int]
        lib.gg_rmat.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_uint64, ctypes.c_int, i32p, i32p, ctypes.c_int]
        lib.gg_chunglu.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                   ctypes.c_int, i32p, i32p, ctypes.c_int]
        lib.gg_chunglu_num_edges.argtypes = [ctypes.c_uint32, ctypes.c_double]
        lib.gg_chunglu_num_edges.restype = ctypes.c_int64
        lib.gg_permutation.argtypes = [ctypes.c_uint32, ctypes.c_uint64, i32p]
        lib.gg_draw_pub.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64]
        lib.gg_draw_pub.restype = ctypes.c_uint64
        for f in (lib.gg_er, lib.gg_rmat, lib.gg_chunglu):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _out(num_edges, out):
    if out is None:
        return np.empty(num_edges, np.int32), np.empty(num_edges, np.int32)
    src, dst = out
    assert src.dtype == np.int32 and dst.dtype == np.int32
    assert src.size >= num_edges and dst.size >= num_edges
    return src, dst


def _ptr(a):
    return a.ctypes.data if isinstance(a, np.ndarray) else int(a)


def er(n: int, num_edges: int, seed: int, out=None, threads: int = 0):
    """``num_edges`` uniform endpoint pairs in [0, n) (loops/duplicates kept)."""
    src, dst = _out(num_edges, out)
    rc = _L().gg_er(n, num_edges, seed, _ptr(src), _ptr(dst), threads)
    if rc:
        raise ValueError("gg_er: bad arguments")
    return src[:num_edges], dst[:num_edges]


def rmat(scale: int, edge_factor: int = 16, seed: int = 2, a=0.57, b=0.19, c=0.19,
         permute: bool = True, out=None, threads: int = 0, num_edges: int = None):
    """R-MAT with 2^scale vertices and edge_factor * 2^scale generated pairs
    (or only the first ``num_edges`` pairs of that stream)."""
    if num_edges is None:
        num_edges = edge_factor << scale
    src, dst = _out(num_edges, out)
    rc = _L().gg_rmat(scale, num_edges, a, b, c, seed, int(permute), _ptr(src), _ptr(dst), threads)
    if rc:
        raise ValueError("gg_rmat: bad arguments (rc=%d)" % rc)
    return src[:num_edges], dst[:num_edges]


def chunglu_num_edges(n: int, mean_deg: float) -> int:
    return int(_L().gg_chunglu_num_edges(n, mean_deg))


def chunglu(n: int, gamma: float, mean_deg: float, seed: int, permute: bool = True,
            out=None, threads: int = 0):
    """Chung-Lu power-law graph with n*mean_deg/2 drawn endpoint pairs."""
    num_edges = chunglu_num_edges(n, mean_deg)
    src, dst = _out(num_edges, out)
    rc = _L().gg_chunglu(n, gamma, mean_deg, seed, int(permute), _ptr(src), _ptr(dst), threads)
    if rc:
        raise ValueError("gg_chunglu: bad arguments (rc=%d)" % rc)
    return src[:num_edges], dst[:num_edges]


def permutation(n: int, seed: int) -> np.ndarray:
    p = np.empty(n, np.int32)
    _L().gg_permutation(n, seed, p.ctypes.data)
    return p


def draw(seed: int, stream: int, k: int) -> int:
    """Counter-based 64-bit draw k of stream ``stream`` under ``seed``."""
    return int(_L().gg_draw_pub(seed, stream, k))


# ----------------------------------------------------------------- recipes
def er_16k():
    """Erdos-Renyi, n = 16384, 262144 uniform pairs, seed 1."""
    n = 16384
    s, d = er(n, 262144, seed=1)
    return n, s, d


def rmat_cfg(scale: int, seed: int, out=None):
    """R-MAT scale s, edge factor 16, (.57,.19,.19,.05), permuted ids."""
    s, d = rmat(scale, 16, seed, out=out)
    return 1 << scale, s, d


def batch_params(num_graphs: int = 4096, seed: int = 6, n_lo: int = 256, n_hi: int = 65536,
                 d_lo: float = 4.0, d_hi: float = 64.0):
    """Per-graph (n_i, d_i, seed_i): n log-uniform in [n_lo, n_hi], d uniform in
    [d_lo, d_hi], seed_i = draw 2 of stream 2^62 + i under ``seed``."""
    ns = np.empty(num_graphs, np.int32)
    ds = np.empty(num_graphs, np.float64)
    seeds = np.empty(num_graphs, np.uint64)
    lo, hi = math.log(n_lo), math.log(n_hi)
    for i in range(num_graphs):
        st = (1 << 62) + i
        u0 = (draw(seed, st, 0) >> 11) * (1.0 / (1 << 53))
        u1 = (draw(seed, st, 1) >> 11) * (1.0 / (1 << 53))
        ns[i] = min(n_hi, max(n_lo, int(round(math.exp(lo + (hi - lo) * u0)))))
        ds[i] = d_lo + (d_hi - d_lo) * u1
        seeds[i] = draw(seed, st, 2)
    return ns, ds, seeds


def batch(num_graphs: int = 4096, seed: int = 6, gamma: float = 2.5, **kw):
    """Concatenated Chung-Lu edge lists with local ids.

    Returns (nv[G] int32, edge_ofs[G+1] int64, src, dst)."""
    ns, ds, seeds = batch_params(num_graphs, seed, **kw)
    counts = np.array([chunglu_num_edges(int(n), float(d)) for n, d in zip(ns, ds)], np.int64)
    ofs = np.zeros(num_graphs + 1, np.int64)
    np.cumsum(counts, out=ofs[1:])
    src = np.empty(int(ofs[-1]), np.int32)
    dst = np.empty(int(ofs[-1]), np.int32)
    for i in range(num_graphs):
        a, b = int(ofs[i]), int(ofs[i + 1])
        chunglu(int(ns[i]), gamma, float(ds[i]), int(seeds[i]), out=(src[a:b], dst[a:b]))
    return ns, ofs, src, dst


# ------------------------------------------------------------ closed forms
def _pairs(edges):
    e = np.asarray(edges, np.int64).reshape(-1, 2)
    return e[:, 0].astype(np.int32), e[:, 1].astype(np.int32)


def complete(n: int):
    """K_n: C(n,3) triangles, C(n-1,2) per vertex."""
    iu = np.triu_indices(n, 1)
    return n, iu[0].astype(np.int32), iu[1].astype(np.int32)


def wheel(rim: int):
    """Hub 0 joined to an n-cycle 1..n (n >= 4): n triangles; hub n, rim 2."""
    e = [(0, i) for i in range(1, rim + 1)] + [(i, i % rim + 1) for i in range(1, rim + 1)]
    s, d = _pairs(e)
    return rim + 1, s, d


def complete_multipartite(*sizes):
    """K_{a,b,c,...}; for three parts a*b*c triangles."""
    part = np.repeat(np.arange(len(sizes)), sizes)
    n = int(sum(sizes))
    iu = np.triu_indices(n, 1)
    keep = part[iu[0]] != part[iu[1]]
    return n, iu[0][keep].astype(np.int32), iu[1][keep].astype(np.int32)


def random_bipartite(a: int, b: int, p: float, seed: int):
    """Random bipartite graph (no triangles)."""
    rng = np.random.default_rng(seed)
    m = rng.random((a, b)) < p
    i, j = np.nonzero(m)
    return a + b, i.astype(np.int32), (j + a).astype(np.int32)


def friendship(k: int):
    """Friendship graph F_k: k triangles sharing vertex 0."""
    e = []
    for t in range(k):
        x, y = 1 + 2 * t, 2 + 2 * t
        e += [(0, x), (0, y), (x, y)]
    s, d = _pairs(e)
    return 2 * k + 1, s, d


def cycle(n: int):
    s, d = _pairs([(i, (i + 1) % n) for i in range(n)])
    return n, s, d


def star(n: int):
    s, d = _pairs([(0, i) for i in range(1, n)])
    return n, s, d


def random_tree(n: int, seed: int):
    rng = np.random.default_rng(seed)
    parent = np.array([rng.integers(0, i) for i in range(1, n)], np.int32)
    return n, np.arange(1, n, dtype=np.int32), parent
