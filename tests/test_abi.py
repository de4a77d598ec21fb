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


def test_null_handles_and_bad_sizes_are_rejected_before_any_device_work():
    """Every entry point checks its handles and sizes first: NULL contexts,
    graphs, batches and servers, and out-of-range sizes, give DSG_ERR_INVALID
    (the void calls return) without touching a device, so this runs on the
    CPU.  The argument types are the binding's."""
    from paper_2311_04333_gb300 import _dsg
    L, BAD = _dsg.LIB, _dsg.DSG_ERR_INVALID
    res, info = _dsg.dsg_result(), _dsg.dsg_prune_info()
    bres, sres = _dsg.dsg_batch_result(), _dsg.dsg_server_result()
    out, km, tk = ctypes.c_void_p(), ctypes.c_int64(), ctypes.c_uint64()
    one = (ctypes.c_int64 * 2)(0, 0)
    buf = (ctypes.c_int32 * 8)()
    codes = {
        "create(out=NULL)": L.dsg_create(0, None, None),
        "upload_csr(ctx=NULL)": L.dsg_upload_csr(None, 1, one, None, 0, ctypes.byref(out)),
        "graph_info(NULL)": L.dsg_graph_info(None, None, None, None),
        "run(NULL)": L.dsg_run(None, 0, 1, 0, 1, None, ctypes.byref(res)),
        "coreness(NULL)": L.dsg_coreness(None, buf, ctypes.byref(km), 0),
        "apx_coreness(NULL)": L.dsg_apx_coreness(None, 3, 2, buf, ctypes.byref(km), 0),
        "run_pruned(NULL)": L.dsg_run_pruned(None, 0, 1, 0, 1, ctypes.byref(res), ctypes.byref(info)),
        "run_pruned_apx(NULL)": L.dsg_run_pruned_apx(None, 0, 1, 0, 1, 3, 2, ctypes.byref(res), ctypes.byref(info)),
        "run_pruned_apx_exact(NULL)": L.dsg_run_pruned_apx_exact(None, 0, 1, 0, 1, 3, 2, ctypes.byref(res),
                                                                 ctypes.byref(info)),
        "set_profiling(NULL)": L.dsg_set_profiling(None, 1),
        "get_stats(NULL)": L.dsg_get_stats(None, None, None, None, 0),
        "get_peel_stats(NULL)": L.dsg_get_peel_stats(None, None, None, None, 0),
        "upload_batch(ctx=NULL)": L.dsg_upload_batch(None, 1, one, None, None, 0, ctypes.byref(out)),
        "batch_info(NULL)": L.dsg_batch_info(None, None, None, None),
        "run_batch(NULL)": L.dsg_run_batch(None, 0, None, None, None, 0, ctypes.byref(bres)),
        "set_batch_tuning(NULL)": L.dsg_set_batch_tuning(None, 0, 0),
        "server_create(slots=0)": L.dsg_server_create(0, 0, 0, ctypes.byref(out)),
        "server_create(budget<0)": L.dsg_server_create(0, 2, -1, ctypes.byref(out)),
        "server_submit(NULL)": L.dsg_server_submit(None, 1, one, None, 0, 1, 0, 1, ctypes.byref(tk)),
        "server_wait(NULL)": L.dsg_server_wait(None, 1, 0, ctypes.byref(sres), None, None),
        "server_stats(NULL)": L.dsg_server_stats(None, None, None, None, None, None),
        "debug_set(spin limit, ctx=NULL)": L.dsg_debug_set(None, _dsg.DSG_DEBUG_SPIN_LIMIT, 10),
        "debug_set(unknown knob)": L.dsg_debug_set(None, 99, 0),
        "debug_set(alloc countdown < 0)": L.dsg_debug_set(None, _dsg.DSG_DEBUG_FAIL_ALLOC, -1),
        "noalloc(n=0)": L.dsg_densest_suffix_noalloc(buf, buf, 0, 0, one, None),
        "noalloc(n too large)": L.dsg_densest_suffix_noalloc(buf, buf, _dsg.DSG_NOALLOC_MAX_VERTICES + 1, 0, one,
                                                             None),
        "noalloc(m >= 2^48)": L.dsg_densest_suffix_noalloc(buf, buf, 4, 1 << 48, one, None),
        "noalloc(NULL loads)": L.dsg_densest_suffix_noalloc(None, buf, 4, 0, one, None),
    }
    wrong = {k: v for k, v in codes.items() if v != BAD}
    assert not wrong, wrong
    assert out.value is None
    L.dsg_destroy(None)
    L.dsg_free_graph(None)
    L.dsg_free_batch(None)
    L.dsg_server_destroy(None)
    assert L.dsg_last_error(None) == b"no context"


def test_header_is_plain_c_and_a_c_program_links_against_the_library(tmp_path):
    """include/dsg.h compiles as C99 with every warning an error, and a C
    program built against it links with libdsg.so and calls entry points
    that need no device."""
    import subprocess
    import paper_2311_04333_gb300 as dsg
    src = tmp_path / "use_dsg.c"
    src.write_text(
        "#include <stdio.h>\n#include \"dsg.h\"\n"
        "int main(void) {\n"
        "    int64_t n = -1;\n"
        "    dsg_ctx *ctx = 0;\n"
        "    if (dsg_graph_info(0, &n, 0, 0) != DSG_ERR_INVALID || n != -1) return 1;\n"
        "    if (dsg_create(0, 0, 0) != DSG_ERR_INVALID) return 2;\n"
        "    (void)ctx;\n"
        "    printf(\"%s\\n\", dsg_last_error(0));\n"
        "    return 0;\n"
        "}\n")
    exe = tmp_path / "use_dsg"
    lib = dsg.LIB_PATH
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), lib, "-Wl,-rpath," + os.path.dirname(lib)], check=True)
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert run.returncode == 0 and run.stdout.strip() == "no context", (run.returncode, run.stdout, run.stderr)
