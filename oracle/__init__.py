"""ORACLE for the AOT hot path -- test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import this package.  It shares
no code with the CUDA path (``paper_2006_11494_gb300``) and neither imports
the other.  The arithmetic lives in ``aot_oracle.c`` (plain single-threaded C,
exact uint64 counts) and in ``mlp.py`` (numpy float64); this file only loads
the C library and marshals numpy arrays.

Functions whose parity is not pinned by an independent check are listed in
the header of the module that defines them (none in this file).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aot_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

ORDER_DESC = 0  # eta: degree non-increasing, ties by smaller id
ORDER_ASC = 1   # eta: degree non-decreasing, ties by smaller id
ORDER_DEGEN = 2  # eta: degeneracy order (peeling round, then id)

OK, ERR_ARG, ERR_RANGE, ERR_NOMEM = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (plain -O2; OpenMP for the *_par paths)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", _SRC,
                               "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.og_new.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, ctypes.POINTER(ctypes.c_int)]
        lib.og_new.restype = P
        lib.og_free.argtypes = [P]
        lib.og_n.argtypes = [P]
        lib.og_n.restype = ctypes.c_int32
        lib.og_m.argtypes = [P]
        lib.og_m.restype = ctypes.c_int64
        lib.og_degrees.argtypes = [P, P]
        lib.og_copy.argtypes = [P, P, P]
        lib.og_count.argtypes = [P, P]
        lib.og_count.restype = ctypes.c_uint64
        lib.og_vertex_count.argtypes = [P, ctypes.c_int32]
        lib.og_vertex_count.restype = ctypes.c_uint64
        lib.og_is_triangle.argtypes = [P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32]
        lib.og_is_triangle.restype = ctypes.c_int
        lib.og_eta.argtypes = [P, ctypes.c_int, P, P]
        lib.og_orient.argtypes = [P, ctypes.c_int, P, P, P, P]
        lib.og_orient.restype = ctypes.c_int
        lib.og_costs.argtypes = [P, ctypes.c_int, P]
        lib.og_costs.restype = ctypes.c_int
        lib.og_work.argtypes = [P, ctypes.c_int, P, P]
        lib.og_work.restype = ctypes.c_int
        lib.og_list_ids.argtypes = [P, P, ctypes.c_uint64]
        lib.og_list_ids.restype = ctypes.c_uint64
        lib.og_list_canonical.argtypes = [P, ctypes.c_int, P, ctypes.c_uint64]
        lib.og_list_canonical.restype = ctypes.c_uint64
        lib.og_stream_vertex_counts.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P,
                                                ctypes.c_int32, P, P]
        lib.og_stream_vertex_counts.restype = ctypes.c_int
        lib.og_degeneracy.argtypes = [P, P, P]
        lib.og_degeneracy.restype = ctypes.c_int
        lib.og_work_rule.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P]
        lib.og_work_rule.restype = ctypes.c_int
        lib.og_costs_noclip.argtypes = [P, ctypes.c_int, P]
        lib.og_costs_noclip.restype = ctypes.c_int
        lib.og_threads.argtypes = [ctypes.c_int]
        lib.og_threads.restype = ctypes.c_int
        lib.og_new_par.argtypes = [ctypes.c_int32, ctypes.c_int64, P, P, ctypes.POINTER(ctypes.c_int),
                                   ctypes.c_int]
        lib.og_new_par.restype = P
        lib.og_count_par.argtypes = [P, P, ctypes.c_int]
        lib.og_count_par.restype = ctypes.c_uint64
        lib.og_list_canonical_par.argtypes = [P, ctypes.c_int, P, ctypes.c_uint64, ctypes.c_int]
        lib.og_list_canonical_par.restype = ctypes.c_uint64
        _lib = lib
    return _lib


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


class OracleError(ValueError):
    def __init__(self, status):
        super().__init__({ERR_ARG: "invalid argument", ERR_RANGE: "vertex id out of range",
                          ERR_NOMEM: "out of memory"}.get(status, "oracle status %d" % status))
        self.status = status


class Graph:
    """The cleaned simple graph of an undirected edge list (loops dropped,
    duplicate and reversed pairs merged, ids checked against [0, n))."""

    def __init__(self, n: int, src, dst, threads: int = None):
        """threads=None: the serial og_new; an int: og_new_par with that many
        threads (0 = all host cores)."""
        src, dst = _i32(src), _i32(dst)
        if src.shape != dst.shape:
            raise OracleError(ERR_ARG)
        st = ctypes.c_int(0)
        if threads is None:
            self._h = _L().og_new(int(n), int(src.size), src.ctypes.data, dst.ctypes.data,
                                  ctypes.byref(st))
        else:
            self._h = _L().og_new_par(int(n), int(src.size), src.ctypes.data, dst.ctypes.data,
                                      ctypes.byref(st), int(threads))
        if st.value != OK:
            raise OracleError(st.value)
        self.n = int(n)
        self.m = int(_L().og_m(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _L().og_free(h)
            self._h = None

    def degrees(self) -> np.ndarray:
        d = np.empty(self.n, np.int32)
        _L().og_degrees(self._h, d.ctypes.data)
        return d

    def csr(self):
        off = np.empty(self.n + 1, np.int64)
        adj = np.empty(2 * self.m, np.int32)
        _L().og_copy(self._h, off.ctypes.data, adj.ctypes.data)
        return off, adj

    def count(self) -> int:
        return int(_L().og_count(self._h, None))

    def count_per_vertex(self):
        t = np.empty(self.n, np.uint64)
        total = int(_L().og_count(self._h, t.ctypes.data))
        return total, t

    def count_par(self, threads: int = 0) -> int:
        """T by the parallel CF edge iterator (0 threads = all host cores)."""
        T = int(_L().og_count_par(self._h, None, int(threads)))
        if T == (1 << 64) - 1:
            raise OracleError(ERR_NOMEM)
        return T

    def count_per_vertex_par(self, threads: int = 0):
        t = np.empty(self.n, np.uint64)
        total = int(_L().og_count_par(self._h, t.ctypes.data, int(threads)))
        if total == (1 << 64) - 1:
            raise OracleError(ERR_NOMEM)
        return total, t

    def list_canonical_par(self, order: int = ORDER_DESC, threads: int = 0) -> np.ndarray:
        total = int(_L().og_list_canonical_par(self._h, order, None, 0, int(threads)))
        if total == (1 << 64) - 1:
            raise OracleError(ERR_NOMEM)
        out = np.empty((max(total, 1), 3), np.int32)
        got = int(_L().og_list_canonical_par(self._h, order, out.ctypes.data, total, int(threads)))
        if got != total:
            raise OracleError(ERR_NOMEM)
        return out[:total]

    def vertex_count(self, v: int) -> int:
        return int(_L().og_vertex_count(self._h, int(v)))

    def is_triangle(self, a, b, c) -> bool:
        return bool(_L().og_is_triangle(self._h, int(a), int(b), int(c)))

    def eta(self, order: int = ORDER_DESC):
        rank = np.empty(self.n, np.int32)
        perm = np.empty(self.n, np.int32)
        _L().og_eta(self._h, order, rank.ctypes.data, perm.ctypes.data)
        return rank, perm

    def orient(self, order: int = ORDER_DESC):
        """(rank[n], perm[n], out_off[n+1] int64, out_adj[m]) in rank space."""
        rank = np.empty(self.n, np.int32)
        perm = np.empty(self.n, np.int32)
        off = np.empty(self.n + 1, np.int64)
        adj = np.empty(max(self.m, 1), np.int32)
        st = _L().og_orient(self._h, order, rank.ctypes.data, perm.ctypes.data,
                            off.ctypes.data, adj.ctypes.data)
        if st:
            raise OracleError(st)
        return rank, perm, off, adj[: self.m]

    def costs(self, order: int = ORDER_DESC) -> dict:
        out = np.zeros(5, np.uint64)
        st = _L().og_costs(self._h, order, out.ctypes.data)
        if st:
            raise OracleError(st)
        return {"sum_deg_head": int(out[0]), "sum_min": int(out[1]), "sum_cf": int(out[2]),
                "walk": int(out[3]), "positive": int(out[4])}

    def work(self, order: int = ORDER_DESC):
        """Per-pivot (rank space) item counts and walk sums of Algorithm 3."""
        items = np.empty(self.n, np.uint32)
        walk = np.empty(self.n, np.uint64)
        st = _L().og_work(self._h, order, items.ctypes.data, walk.ctypes.data)
        if st:
            raise OracleError(st)
        return items, walk

    def work_rule(self, rule: int, order: int = ORDER_DESC):
        """Per-pivot items and walks for rule 0 (Algorithm 3 with the clip),
        1 (Algorithm 3 as printed) or 2 (every edge walked from its tail)."""
        items = np.empty(self.n, np.uint32)
        walk = np.empty(self.n, np.uint64)
        st = _L().og_work_rule(self._h, order, int(rule), items.ctypes.data, walk.ctypes.data)
        if st:
            raise OracleError(st)
        return items, walk

    def degeneracy(self):
        """(round[n], level[n]) of the level-by-level peeling; level = core number."""
        rnd = np.empty(self.n, np.int32)
        lvl = np.empty(self.n, np.int32)
        st = _L().og_degeneracy(self._h, rnd.ctypes.data, lvl.ctypes.data)
        if st:
            raise OracleError(st)
        return rnd, lvl

    def walk_noclip(self, order: int = ORDER_DESC) -> int:
        out = np.zeros(1, np.uint64)
        st = _L().og_costs_noclip(self._h, order, out.ctypes.data)
        if st:
            raise OracleError(st)
        return int(out[0])

    def list_ids(self) -> np.ndarray:
        total = int(_L().og_list_ids(self._h, None, 0))
        out = np.empty((max(total, 1), 3), np.int32)
        _L().og_list_ids(self._h, out.ctypes.data, total)
        return out[:total]

    def list_canonical(self, order: int = ORDER_DESC) -> np.ndarray:
        total = int(_L().og_list_canonical(self._h, order, None, 0))
        out = np.empty((max(total, 1), 3), np.int32)
        _L().og_list_canonical(self._h, order, out.ctypes.data, total)
        return out[:total]


def host_threads(threads: int = 0) -> int:
    """Threads the parallel paths use (0 = all host cores)."""
    return int(_L().og_threads(int(threads)))


def stream_vertex_counts(n: int, src, dst, verts) -> np.ndarray:
    """t(v) for the sampled ``verts`` straight from a raw edge list."""
    src, dst = _i32(src), _i32(dst)
    verts = _i32(verts)
    out = np.empty(verts.size, np.uint64)
    st = _L().og_stream_vertex_counts(int(n), int(src.size), src.ctypes.data, dst.ctypes.data,
                                      int(verts.size), verts.ctypes.data, out.ctypes.data)
    if st:
        raise OracleError(st)
    return out
