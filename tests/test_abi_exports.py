"""The C-ABI library builds for sm_103a and exports every symbol the header declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(hufield_[a-z_]+)\s*\(", src))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared()
    for must in ("hufield_generate", "hufield_threshold", "hufield_spectrum", "hufield_pipeline",
                 "hufield_plan_create", "hufield_workspace_bytes", "hufield_mlp_forward", "hufield_mlp_backward",
                 "hufield_mlp_adam"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2509_08675_gb300 import builder

    lib = ctypes.CDLL(builder.build())
    missing = [n for n in declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_a_gpu():
    from paper_2509_08675_gb300 import builder

    lib = ctypes.CDLL(builder.build())
    lib.hufield_status_string.restype = ctypes.c_char_p
    assert lib.hufield_status_string(0) == b"ok"
    assert lib.hufield_status_string(3) == b"workspace too small"
    assert lib.hufield_status_string(7).startswith(b"the filter passes no power")
    assert lib.hufield_status_string(99) == b"unknown status"
    lib.hufield_workspace_bytes.restype = ctypes.c_size_t
    assert lib.hufield_workspace_bytes(None, 0, 0) == 0


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    import importlib.util

    spec = importlib.util.spec_from_file_location(
        "hufield_nolib", os.path.join(ROOT, "paper_2509_08675_gb300", "hufield.py"))
    mod = importlib.util.module_from_spec(spec)
    import platform
    import sys

    monkeypatch.setitem(sys.modules, "hufield_nolib", mod)

    monkeypatch.setattr(platform, "machine", lambda: "no-such-arch")
    with pytest.raises(ImportError):
        spec.loader.exec_module(mod)
