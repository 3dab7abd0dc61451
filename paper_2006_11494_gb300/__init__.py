"""GB300-native AOT triangle engine: Python binding of libaot.so.

The binding only marshals arguments: every step of orientation, routing,
intersection, counting and listing runs in the library's CUDA kernels.  The
entry points have the names of the C ABI in ``include/aot.h``; device
buffers are torch CUDA tensors (only their pointers cross the boundary) and
the stream defaults to torch's current stream.

There is no CPU fallback: importing works without a GPU (so the library can
be inspected), but every compute call needs the compiled library and a CUDA
device, and raises otherwise.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libaot.so")

# aot_status
OK, ERR_INVALID_ARG, ERR_VERTEX_RANGE, ERR_OVERFLOW, ERR_WORKSPACE, ERR_CUDA, ERR_TIMEOUT, \
    ERR_DEVICE_CHECK, ERR_NOT_READY = range(9)
# aot_route
ROUTE_PLAIN, ROUTE_LEARNED, ROUTE_PROBE, ROUTE_MERGE, ROUTE_BSEARCH, ROUTE_RANDOM = range(6)
# orientation flags
ETA_DEG_DESC = 0x0
ETA_DEG_ASC = 0x1
FLAG_NO_LIST = 0x2
FLAG_NO_CLIP = 0x4
FLAG_LOCAL_RANDOM = 0x8
FLAG_TAIL_PIVOT = 0x10
ETA_DEGENERACY = 0x20

_lib = None

# name -> (restype, argtypes); mirrors include/aot.h
P, I32, I64, U32, U64, SZ = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                             ctypes.c_uint64, ctypes.c_size_t)
SIGNATURES = {
    "aot_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "aot_version": (ctypes.c_int, []),
    "aot_orient_workspace_size": (ctypes.c_int, [I64, I32, U32, ctypes.POINTER(SZ)]),
    "aot_orient": (ctypes.c_int, [P, P, I64, I32, U32, P, SZ, P, ctypes.POINTER(P)]),
    "aot_graph_costs": (ctypes.c_int, [P, P]),
    "aot_graph_info": (ctypes.c_int, [P, ctypes.POINTER(I32), ctypes.POINTER(I64),
                                      ctypes.POINTER(U64), ctypes.POINTER(U64),
                                      ctypes.POINTER(I32)]),
    "aot_graph_export": (ctypes.c_int, [P, P, P, P, P, P, P, P]),
    "aot_count": (ctypes.c_int, [P, ctypes.c_int, ctypes.POINTER(U64), P]),
    "aot_count_per_vertex": (ctypes.c_int, [P, ctypes.c_int, P, ctypes.POINTER(U64), P]),
    "aot_list": (ctypes.c_int, [P, ctypes.c_int, U64, P, U64, ctypes.POINTER(U64),
                                ctypes.POINTER(U64), P]),
    "aot_graph_bins": (ctypes.c_int, [P, P]),
    "aot_graph_get_tuning": (ctypes.c_int, [P, P]),
    "aot_graph_set_tuning": (ctypes.c_int, [P, P, P]),
    "aot_graph_destroy": (ctypes.c_int, [P]),
    "aot_count_per_vertex_static": (ctypes.c_int, [P, P, I64, I32, P, ctypes.POINTER(U64), P]),
    "aot_graph_set_router": (ctypes.c_int, [P, P]),
    "aot_graph_features": (ctypes.c_int, [P, P, P]),
    "aot_graph_record_costs": (ctypes.c_int, [P, I32, I32, P, P]),
    "aot_mlp_forward": (ctypes.c_int, [P, P, I64, P, P]),
    "aot_mlp_train_workspace_size": (ctypes.c_int, [I32, ctypes.POINTER(SZ)]),
    "aot_mlp_train_step": (ctypes.c_int, [P, P, P, P, I32, ctypes.c_float, P, P, I32, P, SZ, P,
                                          ctypes.POINTER(ctypes.c_float), P]),
    "aot_set_default_tuning": (ctypes.c_int, [P]),
    "aot_get_default_tuning": (ctypes.c_int, [P]),
    "aot_tune": (ctypes.c_int, [P, I32, I32, P, ctypes.POINTER(ctypes.c_float), P]),
    "aot_set_default_router": (ctypes.c_int, [P]),
    "aot_batch_workspace_size": (ctypes.c_int, [I64, I32, I64, ctypes.POINTER(SZ)]),
    "aot_batch": (ctypes.c_int, [P, P, P, P, I32, I64, I64, ctypes.c_int, P, P, P, SZ, P]),
    "aot_batch_tune": (ctypes.c_int, [P, P, P, P, I32, I64, I64, I32, P, P, P, SZ, P]),
    "aot_kernel_launches": (ctypes.c_ulonglong, []),
    "aot_profile_begin": (ctypes.c_int, []),
    "aot_profile_end": (ctypes.c_int, [P, I32, ctypes.POINTER(I32)]),
}


class ProfileEntry(ctypes.Structure):
    """Mirror of aot_profile_entry."""
    _fields_ = [("name", ctypes.c_char * 64), ("launches", ctypes.c_uint64),
                ("total_ms", ctypes.c_double)]


class Tuning(ctypes.Structure):
    """Mirror of aot_tuning."""
    _fields_ = [("warp_max_outdeg", ctypes.c_uint32), ("cta_max_outdeg", ctypes.c_uint32),
                ("cta_threads", ctypes.c_int32), ("hub_bitmaps", ctypes.c_int32),
                ("hub_mode", ctypes.c_int32), ("seg_bits", ctypes.c_uint32),
                ("seg_long", ctypes.c_uint32),
                ("seg_wide", ctypes.c_uint32), ("tile_bits", ctypes.c_uint32),
                ("seg_tail", ctypes.c_uint32), ("seg_threads", ctypes.c_int32),
                ("seg_hash", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class AotError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = status
        msg = aot_status_string(status) if _lib is not None else "status %d" % status
        super().__init__("%s: %s (status %d)" % (where, msg, status))


def lib() -> ctypes.CDLL:
    """Load libaot.so (built in-tree by build.py); raise loudly if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libaot.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(st: int, where: str):
    if st != OK:
        raise AotError(st, where)


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


# ------------------------------------------------------------- C ABI mirror
def aot_status_string(status: int) -> str:
    return lib().aot_status_string(status).decode()


def aot_version() -> int:
    return lib().aot_version()


def aot_orient_workspace_size(num_edges: int, num_vertices: int, flags: int = 0) -> int:
    b = SZ(0)
    _check(lib().aot_orient_workspace_size(num_edges, num_vertices, flags, ctypes.byref(b)),
           "aot_orient_workspace_size")
    return b.value


def aot_orient(src, dst, num_vertices: int, flags: int, workspace, stream=None) -> int:
    """Orient an int32 CUDA edge list; returns the opaque graph handle."""
    assert src.dtype == dst.dtype and str(src.dtype) == "torch.int32"
    h = P(0)
    _check(lib().aot_orient(_ptr(src), _ptr(dst), src.numel(), num_vertices, flags,
                            _ptr(workspace), workspace.numel() * workspace.element_size(),
                            _stream(stream), ctypes.byref(h)), "aot_orient")
    return h.value


def aot_graph_info(handle: int) -> dict:
    n, m, w, s, d = I32(0), I64(0), U64(0), U64(0), I32(0)
    _check(lib().aot_graph_info(handle, ctypes.byref(n), ctypes.byref(m), ctypes.byref(w),
                                ctypes.byref(s), ctypes.byref(d)), "aot_graph_info")
    return {"n": n.value, "m": m.value, "W": w.value, "S": s.value, "max_outdeg": d.value}


class Costs(ctypes.Structure):
    """Mirror of aot_costs."""
    _fields_ = [("walk", ctypes.c_uint64), ("merge", ctypes.c_uint64), ("staged", ctypes.c_uint64),
                ("positive", ctypes.c_uint64), ("items", ctypes.c_uint64)]


def aot_graph_costs(handle: int) -> dict:
    c = Costs()
    _check(lib().aot_graph_costs(handle, ctypes.byref(c)), "aot_graph_costs")
    return {k: getattr(c, k) for k, _ in Costs._fields_}


def aot_graph_export(handle: int, perm=None, rank=None, out_off=None, out_adj=None, items=None,
                     walk=None, stream=None):
    _check(lib().aot_graph_export(handle, _ptr(perm), _ptr(rank), _ptr(out_off), _ptr(out_adj),
                                  _ptr(items), _ptr(walk), _stream(stream)), "aot_graph_export")


def aot_count(handle: int, route: int = ROUTE_PLAIN, stream=None) -> int:
    t = U64(0)
    _check(lib().aot_count(handle, route, ctypes.byref(t), _stream(stream)), "aot_count")
    return t.value


def aot_count_per_vertex(handle: int, route: int, counts, want_total: bool = True, stream=None):
    t = U64(0)
    _check(lib().aot_count_per_vertex(handle, route, _ptr(counts),
                                      ctypes.byref(t) if want_total else None, _stream(stream)),
           "aot_count_per_vertex")
    return t.value if want_total else None


def aot_list(handle: int, route: int, cursor: int, out, cap: int, stream=None):
    """Write triangles [cursor, cursor+k) into out (int32, 3*cap); returns (k, next)."""
    k, nxt = U64(0), U64(0)
    _check(lib().aot_list(handle, route, cursor, _ptr(out), cap, ctypes.byref(k),
                          ctypes.byref(nxt), _stream(stream)), "aot_list")
    return k.value, nxt.value


BIN_NAMES = ("warp", "cta", "hub")


def aot_graph_bins(handle: int) -> dict:
    """{bin name: {pivots, items, walk, staged}} under the current tuning."""
    arr = (U64 * 12)()
    _check(lib().aot_graph_bins(handle, ctypes.cast(arr, P)), "aot_graph_bins")
    return {BIN_NAMES[b]: {"pivots": arr[4 * b], "items": arr[4 * b + 1], "walk": arr[4 * b + 2],
                           "staged": arr[4 * b + 3]} for b in range(3)}


def aot_graph_get_tuning(handle: int) -> Tuning:
    t = Tuning()
    _check(lib().aot_graph_get_tuning(handle, ctypes.byref(t)), "aot_graph_get_tuning")
    return t


def aot_graph_set_tuning(handle: int, tuning: Tuning, stream=None):
    _check(lib().aot_graph_set_tuning(handle, ctypes.byref(tuning), _stream(stream)),
           "aot_graph_set_tuning")


MLP_PARAMS = 4931
MLP_MODEL_BYTES = 10240
VARIANTS = ("probe", "merge", "bsearch")


def aot_graph_set_router(handle: int, model):
    _check(lib().aot_graph_set_router(handle, _ptr(model) if model is not None else None),
           "aot_graph_set_router")


def aot_graph_features(handle: int, feat, stream=None):
    _check(lib().aot_graph_features(handle, _ptr(feat), _stream(stream)), "aot_graph_features")


def aot_graph_record_costs(handle: int, variant: int, cycles, sample_log2: int = 0, stream=None):
    _check(lib().aot_graph_record_costs(handle, variant, sample_log2, _ptr(cycles), _stream(stream)),
           "aot_graph_record_costs")


def aot_mlp_forward(model, x, y, stream=None):
    _check(lib().aot_mlp_forward(_ptr(model), _ptr(x), x.shape[0], _ptr(y), _stream(stream)),
           "aot_mlp_forward")


def aot_mlp_train_workspace_size(batch: int) -> int:
    b = SZ(0)
    _check(lib().aot_mlp_train_workspace_size(batch, ctypes.byref(b)), "aot_mlp_train_workspace_size")
    return b.value


def aot_mlp_train_step(model, master, m1, m2, step: int, lr: float, x, t, workspace,
                       grad_out=None, want_loss: bool = True, stream=None):
    loss = ctypes.c_float(0.0)
    _check(lib().aot_mlp_train_step(_ptr(model), _ptr(master), _ptr(m1), _ptr(m2), step, lr,
                                    _ptr(x), _ptr(t), x.shape[0], _ptr(workspace),
                                    workspace.numel() * workspace.element_size(), _ptr(grad_out),
                                    ctypes.byref(loss) if want_loss else None, _stream(stream)),
           "aot_mlp_train_step")
    return loss.value if want_loss else None


STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


def aot_count_per_vertex_static(src, dst, num_vertices: int, counts=None, stream=None) -> int:
    """Per-vertex count with no device allocation (scratch is a fixed device
    array inside the library); returns T and fills ``counts`` if given."""
    t = U64(0)
    _check(lib().aot_count_per_vertex_static(_ptr(src), _ptr(dst), src.numel(), num_vertices,
                                             _ptr(counts), ctypes.byref(t), _stream(stream)),
           "aot_count_per_vertex_static")
    return t.value


def aot_kernel_launches() -> int:
    return int(lib().aot_kernel_launches())


def aot_profile_begin():
    _check(lib().aot_profile_begin(), "aot_profile_begin")


def aot_profile_end() -> dict:
    """{kernel name: (launches, total_ms)} of the launches since aot_profile_begin."""
    cap = 256
    arr = (ProfileEntry * cap)()
    cnt = I32(0)
    _check(lib().aot_profile_end(ctypes.cast(arr, P), cap, ctypes.byref(cnt)), "aot_profile_end")
    return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms))
            for i in range(min(cnt.value, cap))}


def aot_set_default_tuning(tuning: Tuning):
    _check(lib().aot_set_default_tuning(ctypes.byref(tuning)), "aot_set_default_tuning")


def aot_get_default_tuning() -> Tuning:
    t = Tuning()
    _check(lib().aot_get_default_tuning(ctypes.byref(t)), "aot_get_default_tuning")
    return t


def aot_tune(handle: int, mode: int = 0, reps: int = 2, stream=None):
    """Autotune the graph's launch tuning in place; returns (Tuning, best ms)."""
    t = Tuning()
    ms = ctypes.c_float(0.0)
    _check(lib().aot_tune(handle, mode, reps, ctypes.byref(t), ctypes.byref(ms), _stream(stream)),
           "aot_tune")
    return t, ms.value


def aot_set_default_router(model):
    _check(lib().aot_set_default_router(_ptr(model) if model is not None else None),
           "aot_set_default_router")


def aot_batch_workspace_size(total_edges: int, num_graphs: int, total_vertices: int) -> int:
    b = SZ(0)
    _check(lib().aot_batch_workspace_size(total_edges, num_graphs, total_vertices, ctypes.byref(b)),
           "aot_batch_workspace_size")
    return b.value


def aot_batch(src, dst, edge_ofs, nv, route, tri, vcount, workspace, total_vertices=None,
              stream=None):
    """Counts of a batch of graphs (local ids per graph); fills tri[G] and
    vcount[sum nv] (int64 CUDA tensors holding uint64 counts)."""
    G = nv.numel()
    E = src.numel()
    if total_vertices is None:
        total_vertices = int(nv.sum().item())
    _check(lib().aot_batch(_ptr(src), _ptr(dst), _ptr(edge_ofs), _ptr(nv), G, E, total_vertices,
                           route, _ptr(tri), _ptr(vcount) if total_vertices > 0 else None,
                           _ptr(workspace), workspace.numel() * workspace.element_size(),
                           _stream(stream)), "aot_batch")


def aot_batch_tune(src, dst, edge_ofs, nv, workspace, total_vertices=None, reps: int = 1, stream=None):
    """Autotuned tuning of a batch's union graph: (Tuning, best ms)."""
    G = nv.numel()
    E = src.numel()
    if total_vertices is None:
        total_vertices = int(nv.sum().item())
    t = Tuning()
    ms = ctypes.c_float(0)
    _check(lib().aot_batch_tune(_ptr(src), _ptr(dst), _ptr(edge_ofs), _ptr(nv), G, E, total_vertices,
                                reps, ctypes.byref(t), ctypes.byref(ms), _ptr(workspace),
                                workspace.numel() * workspace.element_size(), _stream(stream)),
           "aot_batch_tune")
    return t, ms.value


def aot_graph_destroy(handle: int):
    if handle:
        _check(lib().aot_graph_destroy(handle), "aot_graph_destroy")


# ------------------------------------------------------- convenience object
class OrientedGraph:
    """Owns a workspace tensor and a graph handle (thin wrapper, no compute)."""

    def __init__(self, src, dst, num_vertices: int, flags: int = 0, stream=None):
        import torch
        self.flags = flags
        nbytes = aot_orient_workspace_size(src.numel(), num_vertices, flags)
        self.workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=src.device)
        self.handle = aot_orient(src, dst, num_vertices, flags, self.workspace, stream)
        self.info = aot_graph_info(self.handle)
        self.n, self.m = self.info["n"], self.info["m"]

    def count(self, route: int = ROUTE_PLAIN, stream=None) -> int:
        return aot_count(self.handle, route, stream)

    def count_per_vertex(self, route: int = ROUTE_PLAIN, stream=None):
        import torch
        t = torch.empty(max(self.n, 1), dtype=torch.int64, device=self.workspace.device)
        total = aot_count_per_vertex(self.handle, route, t, True, stream)
        return total, t[: self.n]

    def list(self, route: int = ROUTE_PLAIN, chunk: int = 1 << 24, stream=None):
        """All triangles in canonical order as an (T, 3) int32 CUDA tensor."""
        import torch
        dev = self.workspace.device
        parts, cursor = [], 0
        buf = torch.empty(3 * chunk, dtype=torch.int32, device=dev)
        while True:
            k, nxt = aot_list(self.handle, route, cursor, buf, chunk, stream)
            if k:
                parts.append(buf[: 3 * k].clone())
            if k < chunk:
                break
            cursor = nxt
        if not parts:
            return torch.empty((0, 3), dtype=torch.int32, device=dev)
        return torch.cat(parts).view(-1, 3)

    def set_tuning(self, stream=None, **kw):
        t = aot_graph_get_tuning(self.handle)
        names = {f[0] for f in Tuning._fields_}
        for k, v in kw.items():
            if k not in names:
                raise TypeError("unknown tuning field %r" % k)
            setattr(t, k, v)
        aot_graph_set_tuning(self.handle, t, stream)

    def export(self, stream=None) -> dict:
        import torch
        dev = self.workspace.device
        n, m = self.n, self.m
        out = {
            "perm": torch.empty(max(n, 1), dtype=torch.int32, device=dev),
            "rank": torch.empty(max(n, 1), dtype=torch.int32, device=dev),
            "out_off": torch.empty(n + 1, dtype=torch.int32, device=dev),
            "out_adj": torch.empty(max(m, 1), dtype=torch.int32, device=dev),
            "items": torch.empty(max(n, 1), dtype=torch.int32, device=dev),
            "walk": torch.empty(max(n, 1), dtype=torch.int64, device=dev),
        }
        aot_graph_export(self.handle, out["perm"], out["rank"], out["out_off"], out["out_adj"],
                         out["items"], out["walk"], stream)
        out["perm"], out["rank"] = out["perm"][:n], out["rank"][:n]
        out["out_adj"], out["items"], out["walk"] = out["out_adj"][:m], out["items"][:n], out["walk"][:n]
        return out

    def close(self):
        if getattr(self, "handle", 0):
            aot_graph_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
