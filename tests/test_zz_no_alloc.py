"""aot_count_per_vertex_static: the entry point for callers that cannot
allocate device memory (its scratch is a fixed device array inside the
library).  Called through the C ABI, its output must equal that of the regular
entry points (aot_orient with a caller workspace + aot_count_per_vertex), on
two calls in a row, since every call reuses the same device array.

This file is named to be collected last, so that a stop at the first failure
has already run every other test; it passes alone in a fresh process too."""
import ctypes

import numpy as np
import pytest

import graphgen as gg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def aot():
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_2006_11494_gb300 as m
    return m


def regular(aot, src, dst, n):
    import torch
    ws = torch.empty(aot.aot_orient_workspace_size(src.numel(), n, aot.FLAG_NO_LIST),
                     dtype=torch.uint8, device="cuda")
    h = aot.aot_orient(src, dst, n, aot.FLAG_NO_LIST, ws)
    cnt = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
    total = aot.aot_count_per_vertex(h, aot.ROUTE_PLAIN, cnt)
    aot.aot_graph_destroy(h)
    return total, cnt[:n].cpu().numpy()


def static_call(aot, src, dst, n, with_counts=True):
    """Direct C-ABI call: the caller passes only inputs and outputs."""
    import torch
    cnt = torch.full((max(n, 1),), -1, dtype=torch.int64, device="cuda")
    t = ctypes.c_uint64(0)
    st = aot.lib().aot_count_per_vertex_static(
        src.data_ptr(), dst.data_ptr(), src.numel(), n,
        cnt.data_ptr() if with_counts else None, ctypes.byref(t),
        torch.cuda.current_stream().cuda_stream)
    return st, t.value, cnt[:n].cpu().numpy()


def test_static_matches_regular_on_two_calls_in_a_row(aot):
    import torch
    cases = [gg.er_16k(), gg.rmat_cfg(12, 3)]
    for n, s, d in cases:  # second call reuses the array the first one left behind
        src = torch.from_numpy(s).cuda()
        dst = torch.from_numpy(d).cuda()
        T_reg, t_reg = regular(aot, src, dst, n)
        st, T_st, t_st = static_call(aot, src, dst, n)
        assert st == aot.OK, aot.aot_status_string(st)
        assert T_st == T_reg
        assert np.array_equal(t_st, t_reg)  # integer counts: exact
        st, T_only, _ = static_call(aot, src, dst, n, with_counts=False)
        assert st == aot.OK and T_only == T_reg


def test_static_rejects_oversized_inputs(aot):
    import torch
    n = 65536
    E = 1_200_000
    src = torch.zeros(E, dtype=torch.int32, device="cuda")
    dst = torch.ones(E, dtype=torch.int32, device="cuda")
    st, _, _ = static_call(aot, src, dst, n)
    assert st == aot.ERR_OVERFLOW
    # still usable afterwards
    n, s, d = gg.complete(20)
    st, T, t = static_call(aot, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda(), n)
    assert st == aot.OK and T == 20 * 19 * 18 // 6 and np.all(t == 19 * 18 // 2)
