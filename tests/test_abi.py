"""The C-ABI library builds, loads, and exports every entry point declared
in include/pj.h (no GPU needed: nothing is called)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pj_[a-z0-9_]+)\s*\((?!\*)", src))
    return names


def test_header_declares_entry_points():
    names = declared()
    for n in ("pj_create", "pj_load_set", "pj_join", "pj_join_async", "pj_tri_dist", "pj_pair_bounds",
              "pj_mlp_train", "pj_load_set_streamed", "pj_get_stats", "pj_last_error",
              "pj_voxel_count", "pj_voxels_read", "pj_voxel_labels_read", "pj_voxel_filter"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2604_19982_gb300 import pj
    lib = ctypes.CDLL(pj.LIB_PATH)
    missing = [n for n in sorted(declared()) if not hasattr(lib, n)]
    assert missing == []


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2604_19982_gb300 import pj
    monkeypatch.setattr(pj, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(pj, "_lib", None)
    try:
        pj.lib()
    except RuntimeError as e:
        assert "no CPU fallback" in str(e)
    else:
        raise AssertionError("binding loaded a library that does not exist")
