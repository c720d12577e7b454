"""Serving loops: continuous batching of initial-conditions requests on one GPU.

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
* overlap: in Server every worker thread drives its own CUDA stream and the
  library call holds no Python lock, so requests that arrive while others are on
  the GPU run concurrently with them; in NativeServer (mg_server_*) one C++
  scheduler thread drives all admitted requests as non-blocking pipelines, each
  on its hierarchy's stream, advancing a request whenever the work it queued last
  has finished;
* each result depends only on its own request: the same kernels on the same
  data, no arithmetic shared between requests, so a result is bit-identical
  alone and in the mix.
"""

import collections
import math
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


def _monotonic_perf_counter():
    info = time.get_clock_info("perf_counter")
    return "CLOCK_MONOTONIC" in info.implementation and "RAW" not in info.implementation


class NativeServer:
    """The native serving runtime (mg_server_*): the same admission by HBM budget
    and per-configuration cache of resident hierarchies as Server, but one C++
    scheduler thread drives every admitted request as a non-blocking pipeline
    (an event query per running request and loop pass) instead of one Python
    thread per request blocking on its stream.  Up to `max_active` requests run
    on the GPU at once.  Results are bit-identical to a solo
    Hierarchy.pipeline(host=True) call."""

    def __init__(self, max_active=16, hbm_budget=32 << 30, keep_outputs=True, workers=None,
                 dropped_sets=2):
        import ctypes
        import torch
        self._ct = ctypes
        self._torch = torch
        self.keep_outputs = keep_outputs
        self.hbm_budget = int(hbm_budget)
        self.max_active = int(workers if workers is not None else max_active)
        self.lib = mg.load_library()
        handle = ctypes.c_void_p()
        st = self.lib.mg_server_create(self.hbm_budget, self.max_active, ctypes.byref(handle))
        if st != 0:
            raise mg.MGError(st, "mg_server_create")
        self.h = handle
        self.lock = threading.Condition()
        self.inflight = {}       # id -> (request, kept buffers)
        self.completed = []
        self.peak_inflight = 0
        self._next_id = 0
        self._stop = False
        self._clock_ok = _monotonic_perf_counter()
        # pinned output sets by leaf shapes, returned here when results are not kept:
        # allocating pinned host memory (cudaHostAlloc; 0.5 GB for a 128^3 + 3 x 128^3
        # request) in the submitting thread delayed the arrivals behind it.  _owned: every
        # set allocated per shapes; once a shape has `dropped_sets` of them, a request
        # whose results are dropped writes into one that may still be in use by another
        # such request (the copies still run in full; nobody reads the values).  With
        # dropped_sets=None every request gets a set of its own (the pool grows to the
        # peak number in flight per shapes): measured steadier under load, since
        # concurrent copies into one set of pages ran slower
        self._pool = collections.defaultdict(list)
        self._owned = collections.defaultdict(list)
        self.dropped_sets = dropped_sets
        self._poller = threading.Thread(target=self._poll_loop, daemon=True)
        self._poller.start()

    def submit(self, req):
        ct = self._ct
        if req.arrival is None:
            req.arrival = time.perf_counter()
        nbytes = mg.workspace_bytes(req.cfg)
        if nbytes == 0:
            raise mg.MGError(1, "invalid configuration: " + mg.validate(req.cfg)[1])
        if nbytes > self.hbm_budget:
            raise mg.MGError(2, "request needs %d bytes, above the HBM budget" % nbytes)
        shapes = _leaf_shapes(req.cfg)
        key = tuple(shapes)
        with self.lock:
            pooled = self._pool[key]
            owned = self._owned[key]
            out = pooled.pop() if pooled else None
            if (out is None and not self.keep_outputs and self.dropped_sets is not None
                    and len(owned) >= self.dropped_sets):
                out = owned[self._next_id % len(owned)]
                shared = True
            else:
                shared = False
        if out is None:
            out = self.output_set(shapes)
            if not self.keep_outputs:   # kept results belong to the caller
                with self.lock:
                    owned.append(out)
        d3 = [s for s in shapes for _ in range(3)]
        arrays = [mg._ptrs(req.deltas, shapes, True), mg._ptrs(out["phi1"], shapes, True),
                  mg._ptrs(out["phi2"], shapes, True), mg._ptrs(out["disp1"], d3, True),
                  mg._ptrs(out["disp2"], d3, True)]
        cast = lambda a: ct.cast(a, ct.POINTER(ct.c_void_p))
        with self.lock:
            rid = self._next_id
            self._next_id += 1
            self.inflight[rid] = (req, None if shared else out, arrays, req.cfg)
            self.peak_inflight = max(self.peak_inflight, len(self.inflight))
        st = self.lib.mg_server_submit(self.h, rid, ct.byref(req.cfg), *[cast(a) for a in arrays])
        if st != 0:
            with self.lock:
                del self.inflight[rid]
            raise mg.MGError(st, "mg_server_submit")

    def output_set(self, shapes):
        """A set of pinned host outputs (phi1, phi2, disp1, disp2) for leaf shapes, all
        views of one pinned allocation (one host mapping for the device per set, instead
        of one per array)."""
        torch = self._torch
        sizes = [math.prod(s) for s in shapes]
        slab = torch.empty(8 * sum(sizes), dtype=torch.float64, pin_memory=True)
        off = [0]

        def take(shape, count):
            out = []
            for _ in range(count):
                n = math.prod(shape)
                out.append(slab[off[0]:off[0] + n].view(*shape))
                off[0] += n
            return out
        return {"phi1": [v for s in shapes for v in take(s, 1)],
                "phi2": [v for s in shapes for v in take(s, 1)],
                "disp1": [v for s in shapes for v in take(s, 3)],
                "disp2": [v for s in shapes for v in take(s, 3)]}

    def reserve_outputs(self, cfg, count):
        """Pre-allocates `count` pooled output sets for requests of configuration cfg
        (used when results are not kept), so that arrivals never wait for pinned
        allocation."""
        shapes = tuple(_leaf_shapes(cfg))
        sets = [self.output_set(shapes) for _ in range(count)]
        with self.lock:
            self._pool[shapes].extend(sets)
            self._owned[shapes].extend(sets)

    def _poll_loop(self):
        buf = (mg.MGServerResult * 64)()
        while True:
            n = self.lib.mg_server_poll(self.h, buf, 64, 0.05)
            if n <= 0:
                if self._stop:
                    return
                continue
            now = time.perf_counter()
            with self.lock:
                for i in range(n):
                    r = buf[i]
                    req, out, _, _ = self.inflight.pop(r.id)
                    req.admitted = r.t_start if self._clock_ok else None
                    req.done = r.t_done if self._clock_ok else now
                    nl = req.cfg.n_levels
                    req.info = (r.info1.as_dict(nl), r.info2.as_dict(nl))
                    if r.status != 0:
                        req.error = mg.MGError(r.status, "request %d: %s"
                                               % (req.id, r.error.decode(errors="replace")))
                    if self.keep_outputs:
                        req.outputs = out
                    else:
                        req.outputs = None
                        if out is not None:   # a set this request had to itself
                            self._pool[tuple(_leaf_shapes(req.cfg))].append(out)
                    self.completed.append(req)
                self.lock.notify_all()

    def set_max_instances(self, n):
        """At most n resident hierarchies per configuration (0: no cap)."""
        st = self.lib.mg_server_set_max_instances(self.h, int(n))
        if st != 0:
            raise mg.MGError(st, "mg_server_set_max_instances")

    def stats(self):
        st = mg.MGServerStats()
        self.lib.mg_server_get_stats(self.h, self._ct.byref(st))
        return st.as_dict()

    def drain(self, timeout=600.0):
        """Wait until every submitted request has completed."""
        end = time.perf_counter() + timeout
        with self.lock:
            while self.inflight and time.perf_counter() < end:
                self.lock.wait(timeout=0.05)
            return not self.inflight

    def close(self):
        """Stops the server: requests not yet started fail, running ones finish;
        results not collected by then are dropped (drain() first to keep them)."""
        if self.h is None:
            return
        self._stop = True
        self._poller.join(timeout=60)
        self.lib.mg_server_destroy(self.h)
        self.h = None


def _leaf_shapes(cfg):
    shapes = [tuple(cfg.base_n)]
    for i in range(cfg.n_levels - 1):
        shapes.append(tuple(cfg.nest_n[i]))
    return shapes


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
