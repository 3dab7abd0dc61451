"""The C-ABI library loads and exports every entry point include/aot.h declares;
host-side argument checks return status codes (no GPU needed, no compute)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(aot_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def aot():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2006_11494_gb300 as m
    return m


def test_every_declared_symbol_is_exported(aot):
    names = declared_symbols()
    assert len(names) >= 9, names
    L = aot.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    # the binding mirrors every declared entry point
    assert set(names) <= set(aot.SIGNATURES) | {"aot_version"}


def test_status_strings(aot):
    assert aot.aot_status_string(aot.OK) == "ok"
    for st in range(1, 9):
        assert aot.aot_status_string(st) not in ("", "unknown status")
    assert aot.aot_status_string(999) == "unknown status"
    assert aot.aot_version() >= 100


def test_workspace_size_queries(aot):
    a = aot.aot_orient_workspace_size(1 << 20, 1 << 16)
    b = aot.aot_orient_workspace_size(1 << 20, 1 << 16, aot.FLAG_NO_LIST)
    c = aot.aot_orient_workspace_size(1 << 21, 1 << 16)
    assert 0 < b < a < c
    assert a % 256 == 0
    assert aot.aot_orient_workspace_size(0, 0) > 0
    with pytest.raises(aot.AotError) as e:
        aot.aot_orient_workspace_size(-1, 10)
    assert e.value.status == aot.ERR_INVALID_ARG
    with pytest.raises(aot.AotError) as e:
        aot.aot_orient_workspace_size(10, 10, 0x80)
    assert e.value.status == aot.ERR_INVALID_ARG
    with pytest.raises(aot.AotError) as e:
        aot.aot_orient_workspace_size(1 << 41, 10)
    assert e.value.status == aot.ERR_OVERFLOW


def test_host_side_argument_checks(aot):
    L = aot.lib()
    P = ctypes.c_void_p
    out = P(0)
    # NULL out pointer, NULL workspace, misaligned workspace: rejected before any CUDA call
    assert L.aot_orient(None, None, 0, 0, 0, None, 0, None, None) == aot.ERR_INVALID_ARG
    assert L.aot_orient(None, None, 0, 0, 0, None, 0, None, ctypes.byref(out)) == aot.ERR_WORKSPACE
    assert L.aot_orient(None, None, 0, 0, 0, 8, 1 << 20, None, ctypes.byref(out)) == aot.ERR_WORKSPACE
    assert L.aot_orient(None, None, 5, 10, 0, 256, 1 << 20, None, ctypes.byref(out)) == aot.ERR_INVALID_ARG
    assert L.aot_graph_info(None, None, None, None, None, None) == aot.ERR_INVALID_ARG
    t = ctypes.c_uint64(0)
    assert L.aot_count(None, 0, ctypes.byref(t), None) == aot.ERR_INVALID_ARG
    assert L.aot_count_per_vertex(None, 0, None, None, None) == aot.ERR_INVALID_ARG
    assert L.aot_list(None, 0, 0, None, 0, None, None, None) == aot.ERR_INVALID_ARG
    assert L.aot_graph_destroy(None) == aot.OK


def test_product_does_not_import_oracle():
    """The CUDA path and the oracle share no code and neither imports the other."""
    pkg = os.path.join(ROOT, "paper_2006_11494_gb300")
    bad = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|#include\s+.*oracle)", re.M)
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".c")):
                text = open(os.path.join(dirpath, f)).read()
                assert not bad.search(text), f
                assert "liboracle" not in text and "aot_oracle" not in text, f
    for f in os.listdir(os.path.join(ROOT, "oracle")):
        if f.endswith((".py", ".c")):
            text = open(os.path.join(ROOT, "oracle", f)).read()
            assert "import paper_2006_11494_gb300" not in text and "aot.h" not in text, f
            assert "libaot" not in text, f


def test_documented_default_tuning_is_the_built_in_one(aot):
    text = open(os.path.join(ROOT, "include", "aot.h")).read()
    m = re.search(r"Built-in defaults:(.*?)\.\s*\n", text, flags=re.S)
    assert m, "the header lists the built-in defaults"
    doc = dict((k, int(v)) for k, v in re.findall(r"(\w+) (\d+)", m.group(1).replace("*", " ")))
    assert doc == aot.aot_get_default_tuning().as_dict()
