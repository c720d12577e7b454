"""Serving loop: continuous batching of initial-conditions requests on one GPU.

A request is one hierarchy's whole step (1LPT, 2LPT, both displacement fields)
with its density delta in pinned host memory; the result comes back to pinned
host memory.  Requests arrive open-loop and are admitted in arrival order as soon
as a worker slot is free and their hierarchy fits the HBM budget:

* admission by HBM footprint: a hierarchy's device bytes are known before it is
  created (mg_workspace_bytes); the server keeps the resident total under the
  budget, evicting idle cached hierarchies (least recently used) when needed;
* device-resident level state: hierarchies are cached by configuration, so a
  request whose geometry was seen before reuses the resident levels and its
  captured CUDA graphs; when requests of one configuration overlap, the cache
  holds several instances of it (budget permitting) so they run concurrently;
* overlap: every worker drives its own CUDA stream and the library call holds
  no Python lock, so requests that arrive while others are on the GPU run
  concurrently with them;
* each result depends only on its own request: the same kernels on the same
  data, no arithmetic shared between requests, so a result is bit-identical
  alone and in the mix.
"""

import collections
import threading
import time

from . import mg


class Request:
    def __init__(self, rid, cfg, deltas, arrival=None):
        self.id = rid
        self.cfg = cfg
        self.deltas = deltas          # list of pinned CPU float64 tensors, base first
        self.arrival = arrival        # perf_counter time the request entered the system
        self.admitted = None
        self.done = None
        self.outputs = None
        self.info = None
        self.error = None

    @property
    def latency(self):
        return None if self.done is None else self.done - self.arrival


def config_key(cfg):
    nests = tuple((tuple(cfg.nest_n[i]), tuple(cfg.nest_off[i])) for i in range(cfg.n_levels - 1))
    return (tuple(cfg.base_n), cfg.box, nests, cfg.order, cfg.precision, cfg.nu1, cfg.nu2,
            cfg.max_cycles, cfg.inner_cycles, cfg.tile_rows, cfg.flags, cfg.tol)


class Admission:
    """HBM-budget bookkeeping of resident hierarchies, keyed by configuration.

    cache: key -> list of entries [handle, bytes, busy] (one per resident
    instance of that configuration).  reserve() hands out an idle cached
    instance, or makes room for a new one by closing idle instances (least
    recently used configuration first); it returns None when the request cannot
    run now."""

    def __init__(self, budget, workspace_bytes=None, close=None):
        self.budget = int(budget)
        self.workspace_bytes = workspace_bytes or mg.workspace_bytes
        self.close_handle = close or (lambda h: h.close())
        self.cache = collections.OrderedDict()
        self.resident = 0
        self.peak = 0
        self.evictions = 0

    def _idle_lru(self):
        for key, entries in self.cache.items():
            for e in entries:
                if not e[2]:
                    return key, e
        return None

    def reserve(self, key, cfg):
        for e in self.cache.get(key, ()):
            if not e[2]:
                e[2] = True
                self.cache.move_to_end(key)
                return e
        need = self.workspace_bytes(cfg)
        while self.resident + need > self.budget:
            victim = self._idle_lru()
            if victim is None:
                return None
            vkey, ventry = victim
            self.cache[vkey].remove(ventry)
            if not self.cache[vkey]:
                del self.cache[vkey]
            if ventry[0] is not None:
                self.close_handle(ventry[0])
            self.resident -= ventry[1]
            self.evictions += 1
        entry = [None, need, True]
        self.cache.setdefault(key, []).append(entry)
        self.cache.move_to_end(key)
        self.resident += need
        self.peak = max(self.peak, self.resident)
        return entry

    def instances(self, key):
        return len(self.cache.get(key, ()))

    def release(self, entry):
        entry[2] = False

    def clear(self):
        for entries in self.cache.values():
            for handle, _, _ in entries:
                if handle is not None:
                    self.close_handle(handle)
        self.cache.clear()
        self.resident = 0


class Server:
    """Continuous-batching server with `workers` concurrent requests at most."""

    def __init__(self, workers=4, hbm_budget=32 << 30, keep_outputs=True):
        import torch
        self.keep_outputs = keep_outputs
        self._torch = torch
        self.hbm_budget = int(hbm_budget)
        self.pending = collections.deque()
        self.admission = Admission(hbm_budget)
        self.lock = threading.Condition()
        self.stop = False
        self.completed = []
        self.peak_inflight = 0
        self.inflight = 0
        self.device = torch.cuda.current_device()
        self.threads = [threading.Thread(target=self._worker, args=(w,), daemon=True)
                        for w in range(workers)]
        for t in self.threads:
            t.start()

    # ---- admission ---------------------------------------------------------
    def submit(self, req):
        if req.arrival is None:
            req.arrival = time.perf_counter()
        nbytes = mg.workspace_bytes(req.cfg)
        if nbytes == 0:
            raise mg.MGError(1, "invalid configuration: " + mg.validate(req.cfg)[1])
        if nbytes > self.hbm_budget:
            raise mg.MGError(2, "request needs %d bytes, above the HBM budget" % nbytes)
        with self.lock:
            self.pending.append(req)
            self.lock.notify_all()

    def _next(self):
        """Under the lock: the first pending request (arrival order) that can run now."""
        for i, req in enumerate(self.pending):
            entry = self.admission.reserve(config_key(req.cfg), req.cfg)
            if entry is not None:
                del self.pending[i]
                return req, entry
        return None, None

    # ---- workers -----------------------------------------------------------
    def _worker(self, w):
        torch = self._torch
        torch.cuda.set_device(self.device)
        stream = torch.cuda.Stream()
        while True:
            with self.lock:
                req, entry = None, None
                while not self.stop:
                    req, entry = self._next()
                    if req is not None:
                        break
                    self.lock.wait(timeout=0.05)
                if req is None:
                    return
                self.inflight += 1
                self.peak_inflight = max(self.peak_inflight, self.inflight)
            req.admitted = time.perf_counter()
            try:
                with torch.cuda.stream(stream):
                    if entry[0] is None:
                        entry[0] = mg.Hierarchy(req.cfg, stream=stream)
                    h = entry[0]
                    h.set_stream(stream)
                    out, i1, i2 = h.pipeline(req.deltas, host=True)
                req.outputs = out if self.keep_outputs else None
                req.info = (i1, i2)
            except Exception as exc:  # the request fails, the server keeps serving
                req.error = exc
            req.done = time.perf_counter()
            with self.lock:
                self.admission.release(entry)
                self.inflight -= 1
                self.completed.append(req)
                self.lock.notify_all()

    def drain(self, timeout=600.0):
        """Wait until every submitted request has completed."""
        end = time.perf_counter() + timeout
        with self.lock:
            while (self.pending or self.inflight) and time.perf_counter() < end:
                self.lock.wait(timeout=0.05)
            return not self.pending and not self.inflight

    def close(self):
        with self.lock:
            self.stop = True
            self.lock.notify_all()
        for t in self.threads:
            t.join(timeout=60)
        self.admission.clear()


def run_open_loop(server, requests, rate, seed=5):
    """Submit requests at Poisson arrival times (mean `rate` per second), wait
    for all; returns the wall time from the first arrival to the last result."""
    import numpy as np
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, len(requests))
    t0 = time.perf_counter()
    at = t0
    for req, gap in zip(requests, gaps):
        at += gap
        now = time.perf_counter()
        if at > now:
            time.sleep(at - now)
        req.arrival = at
        server.submit(req)
    server.drain()
    return max(r.done for r in requests) - t0


def latency_stats(requests):
    import numpy as np
    lat = np.array([r.latency for r in requests if r.latency is not None]) * 1e3
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "count": int(lat.size)}
