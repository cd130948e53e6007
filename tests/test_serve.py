"""Host logic of the serving loop (paper_1607_02573_gb300/serve.py): Poisson
arrivals, request mix, the problem cache under a memory budget and the
first-come-first-served queue clock, with fake problems (no GPU)."""

import numpy as np
import pytest

from paper_1607_02573_gb300 import serve as S


def test_poisson_arrivals_rate_and_order():
    t = S.poisson_arrivals(20000, rate=4.0, seed=3)
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.25) <= 0.01
    # exponential gaps: coefficient of variation 1
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
    # seeded: the same arguments give the same requests
    again = S.make_requests(400, rate=2.0, meshes=["a", "b", "c"], seed=5)
    assert [(r.arrival, r.mesh, r.freq, r.kind, r.n_rhs, r.seed) for r in reqs] == \
           [(r.arrival, r.mesh, r.freq, r.kind, r.n_rhs, r.seed) for r in again]


class _Fake:
    def __init__(self, key, nbytes):
        self.key, self.nbytes, self.closed = key, nbytes, False


def _cache(budget, sizes):
    closed = []

    def make(key):
        return _Fake(key, sizes[key[0]])

    def close(p):
        p.closed = True
        closed.append(p.key)

    return S.ProblemCache(budget, make, lambda p: p.nbytes, close), closed


def test_cache_hits_and_lru_eviction_under_budget():
    cache, closed = _cache(100, {"m1": 40, "m2": 50})
    p1, hit = cache.get(("m1", 1.0))
    assert not hit
    p2, hit = cache.get(("m1", 1.1))
    assert not hit and cache.used() == 80
    assert cache.get(("m1", 1.0)) == (p1, True)          # hit, now most recent
    p3, hit = cache.get(("m2", 1.0))                      # 80 + 50 > 100: evict LRU (m1, 1.1)
    assert not hit and closed == [("m1", 1.1)] and p2.closed
    assert set(cache.entries) == {("m1", 1.0), ("m2", 1.0)} and cache.used() == 90
    assert (cache.hits, cache.misses, cache.evictions) == (1, 3, 1)
    cache.clear()
    assert p1.closed and p3.closed and cache.used() == 0


def test_cache_refuses_a_problem_over_the_budget():
    cache, _ = _cache(100, {"big": 150})
    cache.get(("big", 1.0))          # first build: size unknown, built, then alone over budget
    assert cache.used() == 150
    cache.clear()
    with pytest.raises(MemoryError):
        cache.get(("big", 2.0))      # now known to need 150 > 100


def test_queue_clock_and_summary():
    reqs = [S.Request(rid=i, arrival=a, mesh="m", freq=1.0, kind="forward", n_rhs=32, seed=i)
            for i, a in enumerate([0.0, 1.0, 1.5, 10.0])]
    cache, _ = _cache(10 ** 9, {"m": 1})
    now = [0.0]

    def clock():
        return now[0]

    def run(p, r):
        now[0] += 1.0           # every request takes one second of service
        return r.n_rhs

    recs, summ = S.serve(reqs, cache, run, clock=clock)
    assert [x["wait"] for x in recs] == [0.0, 0.0, 0.5, 0.0]
    assert [x["latency"] for x in recs] == [1.0, 1.0, 1.5, 1.0]
    assert summ["columns"] == 128
    assert summ["rhs_solves_per_s"] == pytest.approx(128 / 11.0)
    assert summ["busy_fraction"] == pytest.approx(4 / 11.0)
    assert (summ["cache_hits"], summ["cache_misses"]) == (3, 1)
