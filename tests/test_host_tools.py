"""Host-side logic of the batch autotuner, the serving workload pool and the
Poisson arrival driver, with the library calls replaced by fakes (CPU only)."""
import json
import time

import numpy as np
import pytest


@pytest.fixture()
def tune(monkeypatch):
    from paper_2311_04333_gb300 import _dsg, tune as t
    calls = []
    knobs = {"thread": 0, "block": 0}

    # a batch of 3,000 graphs and 5e6 edges whose launch takes longer with
    # fewer threads per graph, except for a preferred size, and whose
    # preferred degree knobs are 16 (thread scan) and 4096 (block scan)
    def fake_info(batch):
        return 3000, 10_000_000, 5_000_000

    def fake_tuning(ctx, batch, thread_degree=0, block_degree=0):
        knobs["thread"], knobs["block"] = thread_degree, block_degree

    def fake_run(ctx, batch, variant, T, threads, best, eps_num=None, eps_den=None):
        calls.append((variant, threads, knobs["thread"], knobs["block"]))
        extra = 0.004 * (knobs["thread"] not in (0, 16)) if variant == 0 else 0.004 * (knobs["block"] != 4096)
        time.sleep({256: 0.040, 512: 0.005, 1024: 0.020}[threads] + extra)

    monkeypatch.setattr(_dsg, "dsg_batch_info", fake_info)
    monkeypatch.setattr(_dsg, "dsg_run_batch", fake_run)
    monkeypatch.setattr(_dsg, "dsg_set_batch_tuning", fake_tuning)
    monkeypatch.setattr(t, "_gpu_name", lambda: "fake GPU")
    return t, calls, knobs


def test_shape_class_rounds_up_to_powers_of_two():
    from paper_2311_04333_gb300 import tune as t
    assert t._shape_class(4096, 223_270_804) == "G2^12_m2^28"
    assert t._shape_class(3000, 5_000_000) == "G2^12_m2^23"
    assert t._shape_class(1, 0) == "G2^0_m2^0"


def test_tuner_picks_fastest_and_caches(tune, tmp_path):
    t, calls, knobs = tune
    cache = tmp_path / "c.json"
    rec = t.tune_batch(None, "batch", np.full(3000, 8, np.int32), cache_path=str(cache), reps=2)
    assert rec["threads"] == 512 and rec["thread_degree"] == 16
    # block sizes at the default degree, then the other degrees at 512 threads
    assert {k for k in rec["ms"]} == {"256/32", "512/32", "1024/32", "512/8", "512/16", "512/64", "512/128"}
    assert len(calls) == 7 * (1 + 2)                  # one warm-up and two timed runs each
    assert knobs["thread"] == 16                      # the batch is left tuned to the choice
    stored = json.load(open(cache))
    assert list(stored) == ["fake GPU|G2^12_m2^23|variant0"]
    # a second call is served from the cache (and re-applies it); force re-times
    calls.clear()
    knobs["thread"] = 0
    rec2 = t.tune_batch(None, "batch", None, cache_path=str(cache))
    assert (rec2["threads"], knobs["thread"]) == (512, 16)
    assert calls == []
    t.tune_batch(None, "batch", None, cache_path=str(cache), force=True)
    assert len(calls) == 7 * 2


def test_tuner_keys_by_variant(tune, tmp_path):
    t, calls, knobs = tune
    cache = tmp_path / "c.json"
    t.tune_batch(None, "batch", None, cache_path=str(cache), variant=0)
    rec = t.tune_batch(None, "batch", None, cache_path=str(cache), variant=1, eps_num=np.ones(3000, np.int64),
                       eps_den=np.full(3000, 10, np.int64))
    assert sorted(json.load(open(cache))) == ["fake GPU|G2^12_m2^23|variant0", "fake GPU|G2^12_m2^23|variant1"]
    assert {c[0] for c in calls} == {0, 1}
    assert rec["block_degree"] == 4096 and knobs["block"] == 4096


def test_tuner_ignores_a_broken_cache(tune, tmp_path):
    t, _, _ = tune
    cache = tmp_path / "c.json"
    cache.write_text("{not json")
    assert t.tune_batch(None, "batch", None, cache_path=str(cache))["threads"] == 512
    assert "fake GPU|G2^12_m2^23|variant0" in json.load(open(cache))


def test_request_pool_is_seeded_and_follows_the_recipe():
    from paper_2311_04333_gb300 import serve
    a = serve.request_pool(10, seed=7, m_hi=2e5)
    b = serve.request_pool(10, seed=7, m_hi=2e5)
    for x, y in zip(a, b):
        assert x.n == y.n and np.array_equal(x.off, y.off) and np.array_equal(x.adj, y.adj)
    c = serve.request_pool(10, seed=8, m_hi=2e5)
    assert any(x.m != y.m for x, y in zip(a, c))
    for g in a:
        assert 16 <= g.n and 100 <= g.m <= 4e5          # log-uniform targets in [1e3, 2e5]
        deg = np.diff(g.off)
        assert deg.min() >= 1                           # generators drop isolated vertices


def test_poisson_driver_counts_latency_queueing_and_occupancy(monkeypatch):
    """The serving benchmark's driver against a fake server that finishes
    every request 10 ms after its submission (2 ms queued, 8 ms running) on
    one of three workers: the arrival count follows the rate, the statistics
    cover the requests after the warm-up only, and each worker's occupancy is
    the union of its requests' run intervals over the measured span."""
    from paper_2311_04333_gb300 import _dsg, serve
    import graphgen as gg
    sub = {}

    def fake_submit(server, n, off, adj, variant, T, p, q):
        tk = len(sub) + 1
        sub[tk] = (time.perf_counter(), n)
        return tk

    def fake_wait(server, tk, timeout_ms=-1, loads=None, best_set=None):
        t, n = sub[tk]
        if time.perf_counter() - t < 0.010:
            return None
        return {"status": 0, "latency_ms": 10.0, "queue_ms": 2.0, "run_ms": 8.0, "slot": tk % 3, "n": n}

    monkeypatch.setattr(_dsg, "dsg_server_submit", fake_submit)
    monkeypatch.setattr(_dsg, "dsg_server_wait", fake_wait)
    pool = [gg.er_m(100, 4, s) for s in range(4)]
    rate, seconds, warmup = 300.0, 0.6, 0.2
    r = serve.poisson_run(None, pool, rate, seconds, warmup, seed=3)
    # Poisson count over 0.6 s at 300/s: mean 180, standard deviation about 13
    assert 180 - 6 * 14 <= r["requests"] <= 180 + 6 * 14
    assert len(sub) > r["requests"]                  # the warm-up's requests are left out
    assert r["all_ok"] and r["p50_ms"] == 10.0 and r["p99_ms"] == 10.0 and r["mean_queue_ms"] == 2.0
    span = r["submit_span_s"] + r["drain_s"] - warmup
    assert r["throughput_req_s"] == pytest.approx(r["requests"] / span, rel=0.05)
    occ = r["worker_occupancy"]
    assert set(occ) == {0, 1, 2}
    for slot in occ:
        # a third of the arrivals, 8 ms each, overlaps merged: at most 8 ms x rate / 3 per second
        assert 0.0 < occ[slot] <= min(1.0, 0.008 * rate / 3 * 1.6)
