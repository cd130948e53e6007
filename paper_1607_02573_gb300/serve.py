"""Serving loop for imaging requests on one GPU, with continuous batching.

A request names a resident mesh, a frequency, a transmitter set (rings of 32
antennas) and a kind: a forward solve (S-parameters) or a misfit and
gradient against measurements (forward solve, adjoint solve, per-tet
gradient).  Requests arrive in real time and wait in a queue; a dispatcher
admits them as slots and device memory free up:

* a slot is a host worker thread; every problem (operator and factors of one
  (mesh, frequency)) owns its CUDA stream, so batches running in different
  slots overlap on the device;
* a problem is used by one batch at a time; queued forward requests for the
  same problem are merged into one batch -- their columns solved together
  (the pseudo-block FGMRES keeps every column's Krylov space separate, so each
  request's S is the one it would get alone) -- up to a column limit;
  gradient requests run one per batch (their misfit sums over the batch);
* problems stay resident in a least-recently-used cache under a device-memory
  budget; a problem not built yet is admitted only when its estimated bytes
  (from the mesh's decomposition, before building) fit next to the resident
  ones and the batches in flight, evicting idle problems if needed; one that
  cannot fit even alone is refused.  After a batch the entry's real size is
  taken and the budget restored;
* a queued request can be cancelled until it is dispatched.

Latency is measured on the wall clock from arrival to results on the host.
Nothing here touches the oracle.
"""

import collections
import dataclasses
import threading
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
    """Least-recently-used cache of problems keyed by (mesh, frequency), under
    a device-memory budget, for concurrent use.

    make(key) builds a problem; size(problem) gives its device bytes once built;
    estimate(key) its bytes before building; close(problem) frees it.  Entries
    in use by a batch are pinned.  Not thread-safe by itself: the Server calls
    it under its lock."""

    def __init__(self, budget_bytes, make, size, close, estimate=None):
        self.budget = budget_bytes
        self.make, self.size, self.close = make, size, close
        self.estimate = estimate
        self.entries = collections.OrderedDict()   # key -> [problem or None while building, bytes, pins]
        self.seen = {}                             # mesh -> largest bytes observed
        self.hits = self.misses = self.evictions = 0

    def used(self):
        return sum(e[1] for e in self.entries.values())

    def need(self, key):
        """Bytes a new problem for key is expected to take."""
        est = self.estimate(key) if self.estimate else 0
        return max(int(est), self.seen.get(key[0], 0))

    def _evict_idle(self, limit, keep=None):
        for k in list(self.entries):
            if self.used() <= limit:
                break
            e = self.entries[k]
            if k == keep or e[2] > 0 or e[0] is None:
                continue
            self.entries.pop(k)
            self.close(e[0])
            self.evictions += 1

    def reserve(self, key):
        """Admission: pin an entry for key if the memory allows.  Returns
        "hit", "build" (a placeholder sized by the estimate is reserved, the
        caller builds it with build()), "wait" (not now) or "refuse" (the
        problem cannot fit even alone)."""
        if key in self.entries:
            e = self.entries[key]
            if e[2] > 0 or e[0] is None:
                return "wait"              # one batch per problem at a time
            e[2] += 1
            self.entries.move_to_end(key)
            self.hits += 1
            return "hit"
        need = self.need(key)
        if need > self.budget:
            return "refuse"
        self._evict_idle(self.budget - need)
        if self.used() + need > self.budget:
            return "wait"
        self.entries[key] = [None, need, 1]
        self.misses += 1
        return "build"

    def build(self, key):
        """Build the reserved entry (outside the caller's lock)."""
        return self.make(key)

    def built(self, key, problem):
        self.entries[key][0] = problem

    def release(self, key):
        """Unpin after a batch: take the entry's real size and restore the budget."""
        e = self.entries[key]
        e[2] -= 1
        b = self.size(e[0])
        e[1] = b
        self.seen[key[0]] = max(self.seen.get(key[0], 0), b)
        self._evict_idle(self.budget, keep=key)

    def drop(self, key):
        """Forget a reserved entry whose build failed."""
        e = self.entries.pop(key, None)
        if e is not None and e[0] is not None:
            self.close(e[0])

    def get(self, key):
        """Sequential use (no concurrency): reserve, build if needed, and unpin
        at once.  Returns (problem, hit)."""
        st = self.reserve(key)
        if st == "refuse":
            raise MemoryError(f"a problem on mesh {key[0]} needs {self.need(key)} bytes, over the budget")
        if st == "wait":
            raise MemoryError("the budget is held by problems in use")
        if st == "build":
            self.built(key, self.build(key))
        self.release(key)
        return self.entries[key][0], st == "hit"

    def clear(self):
        for e in self.entries.values():
            if e[0] is not None:
                self.close(e[0])
        self.entries.clear()


class Server:
    """Continuous-batching server (module docstring).

    run_batch(problem, requests) does a batch's work and returns
    {rid: (columns solved, result)}; requests of a forward batch share the
    problem and their columns are solved together.  slots = concurrent
    batches; max_cols = the column limit of a merged forward batch."""

    def __init__(self, cache, run_batch, slots=3, max_cols=160, merge=True, clock=time.perf_counter):
        self.cache, self.run_batch = cache, run_batch
        self.slots, self.max_cols, self.merge = slots, max_cols, merge
        self.clock = clock
        self.lock = threading.Condition()
        self.queue = []               # requests waiting, arrival order
        self.running = 0
        self.closed = False
        self.records = {}
        self.results = {}
        self.cancelled = set()
        self.t0 = None
        self.intervals = []           # (start, end) of every batch
        self.merged = 0
        self.workers = []

    # ---- client side
    def start(self):
        self.t0 = self.clock()
        for i in range(self.slots):
            th = threading.Thread(target=self._worker, name=f"slot{i}", daemon=True)
            th.start()
            self.workers.append(th)

    def now(self):
        return self.clock() - self.t0

    def submit(self, r):
        with self.lock:
            self.records[r.rid] = {"rid": r.rid, "mesh": r.mesh, "kind": r.kind, "n_rhs": r.n_rhs,
                                   "arrival": self.now(), "status": "queued"}
            self.queue.append(r)
            self.lock.notify_all()

    def cancel(self, rid):
        """Remove a queued request; False if it was dispatched already."""
        with self.lock:
            for i, r in enumerate(self.queue):
                if r.rid == rid:
                    self.queue.pop(i)
                    self.records[rid]["status"] = "cancelled"
                    self.cancelled.add(rid)
                    self.lock.notify_all()
                    return True
            return False

    def close(self, wait=True):
        """No more requests: finish the queue, stop the slots."""
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        if wait:
            for th in self.workers:
                th.join()

    # ---- dispatch
    def _take(self):
        """Under the lock: the next admissible batch, as (key, requests, cache
        status), or None.  Requests are taken in arrival order; a request whose
        problem is busy or does not fit yet waits, later ones may go first."""
        for i, r in enumerate(self.queue):
            key = (r.mesh, r.freq)
            st = self.cache.reserve(key)
            if st == "wait":
                continue
            if st == "refuse":
                self.queue.pop(i)
                self.records[r.rid].update(status="refused", end=self.now())
                return self._take()
            batch = [self.queue.pop(i)]
            if self.merge and r.kind == "forward":
                cols = r.n_rhs
                j = i
                while j < len(self.queue):
                    q = self.queue[j]
                    if q.kind == "forward" and (q.mesh, q.freq) == key and cols + q.n_rhs <= self.max_cols:
                        batch.append(self.queue.pop(j))
                        cols += q.n_rhs
                    else:
                        j += 1
            return key, batch, st
        return None

    def _worker(self):
        while True:
            with self.lock:
                job = None
                while True:
                    job = self._take()
                    if job is not None or (self.closed and not self.queue):
                        break
                    self.lock.wait(timeout=0.05)
                if job is None:
                    return
                key, batch, st = job
                self.running += 1
                t_start = self.now()
                for r in batch:
                    self.records[r.rid].update(status="running", start=t_start, batch=len(batch),
                                               cache_hit=st == "hit")
                if len(batch) > 1:
                    self.merged += len(batch) - 1
            try:
                if st == "build":
                    p = self.cache.build(key)
                    with self.lock:
                        self.cache.built(key, p)
                else:
                    p = self.cache.entries[key][0]
                out = self.run_batch(p, batch)
                err = None
            except Exception as e:  # noqa: BLE001 -- reported per request
                out, err = {}, repr(e)
            with self.lock:
                t_end = self.now()
                self.intervals.append((t_start, t_end))
                if key in self.cache.entries and self.cache.entries[key][0] is not None:
                    self.cache.release(key)
                else:
                    self.cache.drop(key)
                for r in batch:
                    rec = self.records[r.rid]
                    if err is None:
                        cols, res = out[r.rid]
                        rec.update(status="done", end=t_end, cols=cols, latency=t_end - rec["arrival"],
                                   service=t_end - t_start, wait=t_start - rec["arrival"])
                        self.results[r.rid] = res
                    else:
                        rec.update(status="failed", end=t_end, error=err)
                self.running -= 1
                self.lock.notify_all()

    # ---- report
    def summary(self):
        done = [x for x in self.records.values() if x["status"] == "done"]
        lat = np.array([x["latency"] for x in done]) if done else np.zeros(1)
        cols = sum(x["cols"] for x in done)
        t_first = min((x["arrival"] for x in self.records.values()), default=0.0)
        t_last = max((x.get("end", 0.0) for x in self.records.values()), default=0.0)
        makespan = max(t_last - t_first, 1e-12)
        # time with at least one batch on the device, and the mean number in flight
        ev = sorted([(a, 1) for a, _ in self.intervals] + [(b, -1) for _, b in self.intervals])
        busy = conc = 0.0
        level, last = 0, None
        for t, d in ev:
            if last is not None and level > 0:
                busy += t - last
                conc += level * (t - last)
            level += d
            last = t
        return {"requests": len(self.records), "done": len(done),
                "cancelled": sum(x["status"] == "cancelled" for x in self.records.values()),
                "refused": sum(x["status"] == "refused" for x in self.records.values()),
                "failed": sum(x["status"] == "failed" for x in self.records.values()),
                "columns": int(cols),
                "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
                "rhs_solves_per_s": cols / makespan, "makespan_s": makespan,
                "busy_fraction": busy / makespan, "mean_batches_in_flight": conc / busy if busy > 0 else 0.0,
                "batches": len(self.intervals), "merged_requests": self.merged,
                "cache_hits": self.cache.hits, "cache_misses": self.cache.misses,
                "evictions": self.cache.evictions}


def replay(requests, server, sleep=time.sleep):
    """Submit requests at their arrival times (real time from the server's
    start), then close the server and wait for the queue to drain."""
    server.start()
    for r in sorted(requests, key=lambda q: q.arrival):
        dt = r.arrival - server.now()
        if dt > 0:
            sleep(dt)
        server.submit(r)
    server.close(wait=True)
    return server.summary()


def device_bytes(problem):
    """Device bytes a problem holds (operator, factors, fields, solver
    workspaces), as the library counts them."""
    return int(problem.device_bytes())
