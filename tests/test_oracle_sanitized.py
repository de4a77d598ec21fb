"""The oracle's pins again, on a copy of oracle.c built with gcc's
undefined-behaviour sanitizer (signed overflow, shifts, out-of-bounds
indexing of fixed arrays, misaligned or null accesses), every finding fatal.
The pins check values; this checks that the C arithmetic producing them is
defined, so that they cannot depend on what one compiler made of undefined
code."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PIN_FILES = ["test_oracle_pins.py", "test_oracle_pruned.py", "test_oracle_apx.py", "test_oracle_apx_exact.py",
             "test_oracle_cross.py", "test_golden.py"]


def test_oracle_pins_under_ubsan(tmp_path):
    so = tmp_path / "liboracle_ubsan.so"
    build = subprocess.run(["gcc", "-O1", "-g", "-std=c11", "-shared", "-fPIC", "-fsanitize=undefined",
                            "-fno-sanitize-recover=all", "-o", str(so), os.path.join(ROOT, "oracle", "oracle.c")],
                           capture_output=True, text=True)
    if build.returncode != 0:
        pytest.skip("gcc cannot build with -fsanitize=undefined here: " + build.stderr.strip()[:200])
    # control: the same flags do stop a program at a signed overflow
    src = tmp_path / "overflow.c"
    src.write_text("long long twice(long long x) { return x * 2; }\n")
    ctl = tmp_path / "liboverflow.so"
    subprocess.run(["gcc", "-O1", "-shared", "-fPIC", "-fsanitize=undefined", "-fno-sanitize-recover=all",
                    "-o", str(ctl), str(src)], check=True)
    probe = subprocess.run([sys.executable, "-c", "import ctypes; f = ctypes.CDLL(%r).twice; "
                            "f.argtypes = [ctypes.c_longlong]; f.restype = ctypes.c_longlong; f(1 << 62)" % str(ctl)],
                           capture_output=True, text=True, timeout=60)
    assert probe.returncode != 0 and "runtime error" in probe.stderr, probe.stderr[-500:]
    env = dict(os.environ, DSG_ORACLE_SO=str(so), UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"]
                         + [os.path.join(ROOT, "tests", f) for f in PIN_FILES],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    tail = (run.stdout + run.stderr)[-3000:]
    assert run.returncode == 0, tail
    assert "runtime error" not in run.stderr, tail
