"""Host-side fault hooks of libdsg, on the CPU: the test-only knobs of
dsg_debug_set and the DSG_FAULT environment variable make the allocation
failure path of dsg_create return DSG_ERR_NOMEM before any device is touched,
and reject what they cannot take.  (The same hooks on the GPU, with uploads
and runs that fail and then succeed, are in test_gpu_faults.py.)"""
import ctypes
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
import ctypes, sys
sys.path.insert(0, {root!r})
import paper_2311_04333_gb300 as dsg
lib = ctypes.CDLL(dsg.LIB_PATH)
lib.dsg_create.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
lib.dsg_debug_set.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int64]
out = ctypes.c_void_p(1)
codes = [lib.dsg_create(0, None, ctypes.byref(out)), out.value]
{extra}
print(codes)
"""


def _probe(env_fault=None, extra=""):
    env = dict(os.environ)
    env.pop("DSG_FAULT", None)
    if env_fault:
        env["DSG_FAULT"] = env_fault
    env["CUDA_VISIBLE_DEVICES"] = ""      # these paths must not need a device
    r = subprocess.run([sys.executable, "-c", PROBE.format(root=ROOT, extra=extra)], env=env,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    return eval(r.stdout.strip().splitlines()[-1])


def test_env_fault_makes_create_fail_with_nomem():
    import paper_2311_04333_gb300 as dsg
    codes = _probe("alloc:1")
    assert codes == [dsg.DSG_ERR_NOMEM, None]


def test_countdown_fires_once():
    import paper_2311_04333_gb300 as dsg
    # the first create fails on its injected allocation; the second gets as
    # far as the (absent) device
    codes = _probe("upload:3,alloc:1", "codes += [lib.dsg_create(0, None, ctypes.byref(out))]")
    assert codes[:2] == [dsg.DSG_ERR_NOMEM, None]
    assert codes[2] == dsg.DSG_ERR_CUDA


def test_debug_set_arms_the_countdown_and_checks_its_arguments():
    import paper_2311_04333_gb300 as dsg
    extra = ("codes += [lib.dsg_debug_set(None, 3, 1), lib.dsg_create(0, None, ctypes.byref(out)),"
             " lib.dsg_debug_set(None, 3, -1), lib.dsg_debug_set(None, 4, 0),"
             " lib.dsg_debug_set(None, 1, 5), lib.dsg_debug_set(None, 2, 1), lib.dsg_debug_set(None, 9, 1)]")
    codes = _probe(None, extra)
    # no fault from the environment: the first create reaches the device check
    assert codes[0] == dsg.DSG_ERR_CUDA
    assert codes[2:] == [dsg.DSG_OK, dsg.DSG_ERR_NOMEM, dsg.DSG_ERR_INVALID, dsg.DSG_OK,
                         dsg.DSG_ERR_INVALID, dsg.DSG_ERR_INVALID, dsg.DSG_ERR_INVALID]
