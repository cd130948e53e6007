"""Host logic of the serving loop (paper_1607_02573_gb300/serve.py): Poisson
arrivals, request mix, the problem cache under a memory budget, and the
continuous-batching server (admission by slots and memory, merging of
forward requests that share a problem, one batch per problem at a time,
overlap of batches, cancellation, refusal), with fake problems (no GPU)."""

import threading
import time

import numpy as np
import pytest

from paper_1607_02573_gb300 import serve as S


def test_poisson_arrivals_rate_and_order():
    t = S.poisson_arrivals(20000, rate=4.0, seed=3)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.25) <= 0.01
    gaps = np.diff(t)
    assert abs(np.std(gaps) / np.mean(gaps) - 1.0) <= 0.05


def test_request_mix():
    reqs = S.make_requests(400, rate=2.0, meshes=["a", "b", "c"], seed=5)
    assert [r.rid for r in reqs] == list(range(400))
    assert {r.mesh for r in reqs} == {"a", "b", "c"}
    f = np.array([r.freq for r in reqs])
    assert f.min() >= 0.8e9 - 1 and f.max() <= 1.2e9 + 1
    assert np.allclose((f - 0.8e9) / 10e6, np.round((f - 0.8e9) / 10e6))
    assert {r.n_rhs for r in reqs} <= {32, 64, 96, 128, 160}
    kinds = [r.kind for r in reqs]
    assert 0.4 < kinds.count("forward") / len(kinds) < 0.6
    again = S.make_requests(400, rate=2.0, meshes=["a", "b", "c"], seed=5)
    assert [(r.arrival, r.mesh, r.freq, r.kind, r.n_rhs, r.seed) for r in reqs] == \
           [(r.arrival, r.mesh, r.freq, r.kind, r.n_rhs, r.seed) for r in again]


class _Fake:
    def __init__(self, key, nbytes):
        self.key, self.nbytes, self.closed = key, nbytes, False
        self.active = 0


def _cache(budget, sizes, estimate=True):
    closed = []

    def make(key):
        return _Fake(key, sizes[key[0]])

    def close(p):
        p.closed = True
        closed.append(p.key)

    est = (lambda key: sizes[key[0]]) if estimate else None
    return S.ProblemCache(budget, make, lambda p: p.nbytes, close, estimate=est), closed


def test_cache_hits_and_lru_eviction_under_budget():
    cache, closed = _cache(100, {"m1": 40, "m2": 50})
    p1, hit = cache.get(("m1", 1.0))
    assert not hit
    p2, hit = cache.get(("m1", 1.1))
    assert not hit and cache.used() == 80
    assert cache.get(("m1", 1.0)) == (p1, True)
    p3, hit = cache.get(("m2", 1.0))                      # 80 + 50 > 100: evict LRU (m1, 1.1) first
    assert not hit and closed == [("m1", 1.1)] and p2.closed
    assert set(cache.entries) == {("m1", 1.0), ("m2", 1.0)} and cache.used() == 90
    assert (cache.hits, cache.misses, cache.evictions) == (1, 3, 1)
    cache.clear()
    assert p1.closed and p3.closed and cache.used() == 0


def test_cache_estimates_before_building_and_refuses_oversized():
    cache, closed = _cache(100, {"m1": 70, "big": 150})
    cache.get(("m1", 1.0))
    # admitting m1 at another frequency needs 70 more bytes: the idle entry is evicted before the build
    st = cache.reserve(("m1", 2.0))
    assert st == "build" and closed == [("m1", 1.0)] and cache.used() == 70
    assert cache.reserve(("big", 1.0)) == "refuse"       # over the budget by its estimate, never built
    assert all(k[0] != "big" for k in cache.entries)


def test_cache_pins_entries_in_use():
    cache, closed = _cache(100, {"m1": 60, "m2": 60})
    assert cache.reserve(("m1", 1.0)) == "build"
    cache.built(("m1", 1.0), cache.build(("m1", 1.0)))
    assert cache.reserve(("m1", 1.0)) == "wait"          # one batch per problem at a time
    assert cache.reserve(("m2", 1.0)) == "wait"          # m1 is pinned: no room
    cache.release(("m1", 1.0))
    assert cache.reserve(("m2", 1.0)) == "build" and closed == [("m1", 1.0)]


def _server(budget, sizes, service, slots=2, merge=True, max_cols=160, log=None):
    cache, _ = _cache(budget, sizes)
    lock = threading.Lock()

    def run_batch(p, batch):
        with lock:
            p.active += 1
            assert p.active == 1, "two batches on one problem"
            if log is not None:
                log.append(("start", [r.rid for r in batch], time.perf_counter()))
        time.sleep(service)
        with lock:
            p.active -= 1
            if log is not None:
                log.append(("end", [r.rid for r in batch], time.perf_counter()))
        return {r.rid: (r.n_rhs * (2 if r.kind == "gradient" else 1), (p.key, r.rid)) for r in batch}

    return S.Server(cache, run_batch, slots=slots, merge=merge, max_cols=max_cols)


def test_server_merges_forward_requests_of_one_problem():
    srv = _server(10 ** 9, {"m": 1}, service=0.05, slots=1)
    reqs = [S.Request(rid=i, arrival=0.0, mesh="m", freq=1.0, kind=k, n_rhs=32, seed=i)
            for i, k in enumerate(["forward", "forward", "gradient", "forward", "gradient"])]
    # all queued before the single slot starts
    srv.t0 = time.perf_counter()
    for r in reqs:
        srv.submit(r)
    srv.start()
    srv.close()
    s = srv.summary()
    assert s["done"] == 5 and s["columns"] == 32 * 3 + 64 * 2
    batch_of = {rid: rec["batch"] for rid, rec in srv.records.items()}
    assert batch_of[0] == batch_of[1] == batch_of[3] == 3          # the three forward requests together
    assert batch_of[2] == batch_of[4] == 1                         # gradients alone
    assert s["batches"] == 3 and s["merged_requests"] == 2
    assert all(srv.results[r.rid] == (("m", 1.0), r.rid) for r in reqs)


def test_server_overlaps_batches_and_respects_memory():
    log = []
    # two problems fit together, three do not
    srv = _server(130, {"a": 60, "b": 60, "c": 60}, service=0.1, slots=3, log=log)
    reqs = [S.Request(rid=i, arrival=0.01 * i, mesh=m, freq=1.0, kind="gradient", n_rhs=32, seed=i)
            for i, m in enumerate(["a", "b", "c"])]
    summ = S.replay(reqs, srv)
    assert summ["done"] == 3
    starts = {tuple(e[1]): e[2] for e in log if e[0] == "start"}
    ends = {tuple(e[1]): e[2] for e in log if e[0] == "end"}
    # a and b overlap on the device; c starts only after one of them released its memory
    assert starts[(1,)] < ends[(0,)]
    assert starts[(2,)] >= min(ends[(0,)], ends[(1,)])
    assert summ["mean_batches_in_flight"] > 1.2
    assert srv.cache.used() <= 130


def test_server_cancel_refuse_and_latency():
    srv = _server(100, {"m": 10, "huge": 1000}, service=0.05, slots=1)
    srv.start()
    srv.submit(S.Request(rid=0, arrival=0.0, mesh="m", freq=1.0, kind="gradient", n_rhs=32, seed=0))
    srv.submit(S.Request(rid=1, arrival=0.0, mesh="m", freq=1.0, kind="gradient", n_rhs=32, seed=1))
    srv.submit(S.Request(rid=2, arrival=0.0, mesh="huge", freq=1.0, kind="forward", n_rhs=32, seed=2))
    cancelled = srv.cancel(1)
    srv.close()
    s = srv.summary()
    assert cancelled and srv.records[1]["status"] == "cancelled"
    assert srv.records[2]["status"] == "refused"
    assert s["done"] == 1 and s["cancelled"] == 1 and s["refused"] == 1
    rec = srv.records[0]
    assert rec["latency"] == pytest.approx(rec["wait"] + rec["service"])
    assert rec["service"] >= 0.05
