"""Serving loop for imaging requests on one GPU.

A request names a resident mesh, a frequency, a transmitter set (32 to 160
antennas in rings of 32) and a kind: a forward solve (S-parameters) or a
misfit and gradient against seeded synthetic measurements (forward solve,
adjoint solve, per-tet gradient).  Requests are served first come first
served; the device runs one request at a time (a request's columns already
fill the GPU).  Assembled and factorised problems stay resident in a cache
keyed by (mesh, frequency), evicted least recently used when admitting a new
one would exceed the device-memory budget.

Arrivals are Poisson.  The loop serves the requests in arrival order on the
device and keeps the queue's clock: a request starts at max(its arrival, the
previous request's completion), so the latency it reports (completion minus
arrival) includes the time it would have waited in the queue.  Nothing here
touches the oracle.
"""

import collections
import dataclasses
import time

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float       # s, from the start of the run
    mesh: str
    freq: float          # Hz
    kind: str            # "forward" or "gradient"
    n_rhs: int
    seed: int


def poisson_arrivals(n, rate, seed):
    """Arrival times (s) of n requests of a Poisson process of the given rate (1/s)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def make_requests(n, rate, meshes, seed, freq_lo=0.8e9, freq_hi=1.2e9, freq_step=10e6, rings=(1, 2, 3, 4, 5)):
    """n requests with Poisson arrivals: mesh uniform over `meshes`, frequency
    uniform on the freq_step grid of [freq_lo, freq_hi], 32 x rings transmitters,
    forward or gradient with probability 1/2 each."""
    rng = np.random.default_rng(seed + 1)
    t = poisson_arrivals(n, rate, seed)
    grid = np.arange(freq_lo, freq_hi + freq_step / 2, freq_step)
    out = []
    for i in range(n):
        out.append(Request(rid=i, arrival=float(t[i]), mesh=str(meshes[rng.integers(len(meshes))]),
                           freq=float(grid[rng.integers(grid.size)]),
                           kind="forward" if rng.random() < 0.5 else "gradient",
                           n_rhs=32 * int(rings[rng.integers(len(rings))]), seed=int(rng.integers(1 << 30))))
    return out


class ProblemCache:
    """Least-recently-used cache of problems keyed by (mesh, frequency).

    make(key) builds a problem; size(problem) gives its device bytes once built;
    close(problem) frees it.  Before building, entries are evicted until the
    bytes in use plus the largest size seen for that mesh fit the budget; after
    building (and after each use, since solve buffers grow), entries other than
    the newest are evicted while the total exceeds the budget."""

    def __init__(self, budget_bytes, make, size, close):
        self.budget = budget_bytes
        self.make, self.size, self.close = make, size, close
        self.entries = collections.OrderedDict()   # key -> [problem, bytes]
        self.seen = {}                             # mesh -> largest bytes observed
        self.hits = self.misses = self.evictions = 0

    def used(self):
        return sum(b for _, b in self.entries.values())

    def _evict_until(self, limit, keep=None):
        for k in list(self.entries):
            if self.used() <= limit:
                break
            if k == keep:
                continue
            p, _ = self.entries.pop(k)
            self.close(p)
            self.evictions += 1

    def get(self, key):
        if key in self.entries:
            self.entries.move_to_end(key)
            self.hits += 1
            return self.entries[key][0], True
        self.misses += 1
        need = self.seen.get(key[0], 0)
        if need > self.budget:
            raise MemoryError(f"a problem on mesh {key[0]} needs {need} bytes, over the budget")
        self._evict_until(self.budget - need)
        p = self.make(key)
        self.entries[key] = [p, self.size(p)]
        self.account(key)
        return p, False

    def account(self, key):
        """Re-measure an entry after use and restore the budget."""
        p = self.entries[key][0]
        b = self.size(p)
        self.entries[key][1] = b
        self.seen[key[0]] = max(self.seen.get(key[0], 0), b)
        self._evict_until(self.budget, keep=key)

    def clear(self):
        for p, _ in self.entries.values():
            self.close(p)
        self.entries.clear()


def serve(requests, cache, run_request, clock=time.perf_counter):
    """Serve requests in arrival order.  run_request(problem, request) does the
    work and returns the number of right-hand sides solved.  Returns per-request
    records and a summary (latency percentiles, RHS-solves/s over the makespan)."""
    recs = []
    t_dev = 0.0   # the queue's clock: completion of the previous request
    for r in sorted(requests, key=lambda q: q.arrival):
        start = max(r.arrival, t_dev)
        t0 = clock()
        p, hit = cache.get((r.mesh, r.freq))
        cols = run_request(p, r)
        cache.account((r.mesh, r.freq))
        service = clock() - t0
        t_dev = start + service
        recs.append({"rid": r.rid, "mesh": r.mesh, "kind": r.kind, "n_rhs": r.n_rhs, "cols": cols,
                     "cache_hit": hit, "wait": start - r.arrival, "service": service,
                     "latency": t_dev - r.arrival})
    lat = np.array([x["latency"] for x in recs])
    cols = sum(x["cols"] for x in recs)
    makespan = t_dev - (min(r.arrival for r in requests) if requests else 0.0)
    summary = {"requests": len(recs), "columns": int(cols),
               "latency_p50_s": float(np.percentile(lat, 50)) if recs else 0.0,
               "latency_p99_s": float(np.percentile(lat, 99)) if recs else 0.0,
               "rhs_solves_per_s": cols / makespan if makespan > 0 else 0.0,
               "busy_fraction": sum(x["service"] for x in recs) / makespan if makespan > 0 else 0.0,
               "cache_hits": cache.hits, "cache_misses": cache.misses, "evictions": cache.evictions}
    return recs, summary


def device_bytes(problem):
    """Device bytes a problem holds (operator, factors, fields, solver
    workspaces), as the library counts them."""
    return int(problem.device_bytes())
