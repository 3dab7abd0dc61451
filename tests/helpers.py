"""Shared helpers for the GPU parity tests (marshalling only)."""
import numpy as np


def to_dev(s, d):
    import torch
    return (torch.from_numpy(np.ascontiguousarray(s, np.int32)).cuda(),
            torch.from_numpy(np.ascontiguousarray(d, np.int32)).cuda())


def gpu_graph(n, s, d, flags=0):
    import paper_2006_11494_gb300 as aot
    src, dst = to_dev(s, d)
    return aot.OrientedGraph(src, dst, n, flags)


def u64(t):
    """int64 CUDA tensor of counts -> numpy uint64."""
    return t.cpu().numpy().astype(np.uint64)
