"""The Python binding's own checks, on the CPU: buffers smaller than what a
C call reads or writes are refused before the call, and correctly sized ones
go through unchanged.  A stand-in for the loaded library records the calls
(no GPU, no kernels): only the binding's marshalling is under test here."""
import ctypes

import numpy as np
import pytest

from paper_2311_04333_gb300 import _dsg


class FakeLib:
    """Answers the info calls with fixed sizes; every other entry point
    records its name and returns DSG_OK (DSG_ERR_INVALID for a NULL graph)."""

    def __init__(self, n=10, G=3, N=30):
        self.n, self.G, self.N = n, G, N
        self.calls = []

    def dsg_graph_info(self, g, pn, pm, pd):
        if g is None:
            return _dsg.DSG_ERR_INVALID
        pn._obj.value = self.n
        return _dsg.DSG_OK

    def dsg_batch_info(self, b, pG, pN, pm):
        pG._obj.value = self.G
        pN._obj.value = self.N
        return _dsg.DSG_OK

    def dsg_last_error(self, ctx):
        return b"from the stand-in"

    def __getattr__(self, name):
        def call(*args):
            self.calls.append(name)
            return _dsg.DSG_ERR_INVALID if name == "dsg_run" and args[0] is None else _dsg.DSG_OK
        return call


@pytest.fixture()
def lib(monkeypatch):
    fake = FakeLib()
    monkeypatch.setattr(_dsg, "LIB", fake)
    return fake


def test_run_buffers_sized_by_the_graph(lib):
    n, T = lib.n, 4
    _dsg.dsg_run(None, 1, 0, T, 0, 1, None, np.zeros(n, np.int64), np.zeros(n, np.int32), np.zeros(3 * T, np.int64))
    assert lib.calls == ["dsg_run"]
    for kw in (dict(loads=np.zeros(n - 1, np.int64)), dict(best_set=np.zeros(n - 1, np.int32)),
               dict(trace=np.zeros(3 * T - 1, np.int64)), dict(init_loads=np.zeros(n - 1, np.int64))):
        with pytest.raises(ValueError, match="entries"):
            _dsg.dsg_run(None, 1, 0, T, **kw)
    assert lib.calls == ["dsg_run"]
    # larger buffers are fine (the call uses the first n entries)
    _dsg.dsg_run(None, 1, 0, T, loads=np.zeros(n + 5, np.int64))
    assert lib.calls == ["dsg_run"] * 2


def test_unknown_graph_is_left_to_the_library(lib):
    with pytest.raises(_dsg.DsgError) as ei:
        _dsg.dsg_run(None, None, 0, 3, loads=np.zeros(1, np.int64))
    assert ei.value.status == _dsg.DSG_ERR_INVALID


def test_pruned_run_and_coreness_buffers(lib):
    n = lib.n
    _dsg.dsg_run_pruned(None, 1, 0, 2, loads=np.zeros(n, np.int64), trace=np.zeros(6, np.int64))
    with pytest.raises(ValueError):
        _dsg.dsg_run_pruned(None, 1, 0, 2, best_set=np.zeros(n - 1, np.int32))
    with pytest.raises(ValueError):
        _dsg.dsg_run_pruned(None, 1, 0, 2, trace=np.zeros(5, np.int64), c=(3, 2))
    _dsg.dsg_coreness(None, 1)                      # allocated by the binding at n entries
    with pytest.raises(ValueError):
        _dsg.dsg_coreness(None, 1, np.zeros(n - 1, np.int32))
    with pytest.raises(ValueError):
        _dsg.dsg_apx_coreness(None, 1, (3, 2), np.zeros(n - 1, np.int32))
    assert lib.calls == ["dsg_run_pruned", "dsg_coreness"]


def test_upload_arrays_cover_the_graph(lib):
    off = np.array([0, 2, 3, 4], np.int64)
    adj = np.array([1, 2, 0, 0], np.int32)
    _dsg.dsg_upload_csr(None, 3, off, adj)
    with pytest.raises(ValueError, match="offsets"):
        _dsg.dsg_upload_csr(None, 4, off, adj)
    with pytest.raises(ValueError, match="adj"):
        _dsg.dsg_upload_csr(None, 3, off, adj[:3])
    _dsg.dsg_server_submit(None, 3, off, adj, 0, 2)
    with pytest.raises(ValueError, match="adj"):
        _dsg.dsg_server_submit(None, 3, off, adj[:2], 0, 2)
    assert lib.calls == ["dsg_upload_csr", "dsg_server_submit"]


def test_batch_buffers_sized_by_the_batch(lib):
    G, N = lib.G, lib.N
    T = np.array([2, 5, 3], np.int32)
    _dsg.dsg_run_batch(None, 1, 0, T, 0, np.zeros(4 * G, np.int64), np.zeros(N, np.int64),
                       np.zeros(N, np.int32), np.zeros(3 * G * 5, np.int64))
    assert lib.calls == ["dsg_run_batch"]
    bad = [dict(T=T[:2]), dict(best=np.zeros(4 * G - 1, np.int64)), dict(loads=np.zeros(N - 1, np.int64)),
           dict(sets=np.zeros(N - 1, np.int32)), dict(trace=np.zeros(3 * G * 5 - 1, np.int64))]
    for kw in bad:
        args = dict(T=T, best=np.zeros(4 * G, np.int64))
        args.update(kw)
        with pytest.raises(ValueError, match="entries"):
            _dsg.dsg_run_batch(None, 1, 0, args.pop("T"), 0, **args)
    assert lib.calls == ["dsg_run_batch"]
