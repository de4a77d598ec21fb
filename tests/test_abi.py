"""The C ABI library loads and exports every entry point include/dsg.h
declares, and the Python binding mirrors those names (no compute calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dsg_\w+)\s*\(", src))
    return names


def test_header_declares_boundary():
    names = _declared()
    for f in ("dsg_create", "dsg_upload_csr", "dsg_run", "dsg_free_graph", "dsg_destroy",
              "dsg_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol():
    import paper_2311_04333_gb300 as dsg
    lib = ctypes.CDLL(dsg.LIB_PATH)
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, f"libdsg.so lacks {missing}"


def test_binding_has_same_names():
    from paper_2311_04333_gb300 import _dsg
    missing = [n for n in sorted(_declared()) if not hasattr(_dsg, n)]
    assert not missing, f"binding lacks {missing}"


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_2311_04333_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "oracle.c" not in src and "liboracle" not in src, f
