"""The C-ABI library builds, loads and exports every entry point that include/agp.h declares.

Runs without a GPU: only host-side entry points (status strings, version) are called.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "agp.h")).read()
    return sorted(set(re.findall(r"AGP_API\s+[\w\s\*]*?\b(agp_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("agp_build_graph", "agp_graph_info", "agp_graph_destroy", "agp_query", "agp_query_batch",
                     "agp_feature_propagate", "agp_katz_beta", "agp_threshold", "agp_strerror",
                     "agp_last_error_detail"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2106_03058_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_entry_points():
    import paper_2106_03058_gb300 as agp
    L = agp.lib()
    assert L.agp_version() >= 10000
    assert agp._strerror(0) == "AGP_OK" and agp._strerror(1) == "AGP_EINVAL"
    assert agp._strerror(12345) == "AGP_UNKNOWN"
    # NULL handles are rejected with AGP_EINVAL, without touching a device
    assert L.agp_graph_info(None, None, None, None, None, None) == 1
    assert b"NULL" in L.agp_last_error_detail()
    assert L.agp_graph_destroy(None) == 0


def test_no_fallback_when_library_is_missing(tmp_path, monkeypatch):
    """The binding fails loudly if libagp.so cannot be produced: there is no CPU path."""
    import importlib
    import paper_2106_03058_gb300 as agp
    from paper_2106_03058_gb300 import build
    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(build, "_nvcc", lambda: (_ for _ in ()).throw(RuntimeError("nvcc not found")))
    monkeypatch.setattr(agp, "_lib", None)
    with pytest.raises(RuntimeError):
        agp.lib()
    monkeypatch.undo()
    importlib.reload(agp)
