"""ctypes binding of the C ABI in include/mg.h (argument marshalling only).

Every step of the solve runs in the CUDA library libmgic.so; this module only
builds the config struct, passes device pointers of torch tensors and the
current CUDA stream, and turns status codes into exceptions.  There is no CPU
fallback: if the library cannot be loaded, every call raises.
"""

import ctypes
import os

MG_MAX_LEVELS = 16
MG_MAX_HISTORY = 64
MG_FP64 = 0
MG_MIXED = 1
MG_FLAG_NO_GRAPHS = 1
MG_FLAG_NO_TMA = 2
MG_FLAG_TMA_ALL = 4
MG_FLAG_HYBRID = 8
MG_FLAG_DEVICE_LOOP = 16
MG_FLAG_PERSISTENT = 32
MG_FLAG_PAIR_SMOOTHER = 64
_TMA_FLAGS = {"auto": 0, "off": MG_FLAG_NO_TMA, "all": MG_FLAG_TMA_ALL}

STATUS = {0: "MG_OK", 1: "MG_EINVAL", 2: "MG_ENOMEM", 3: "MG_ENOCONV", 4: "MG_ECUDA",
          5: "MG_ETIMEOUT"}

_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class MGConfig(ctypes.Structure):
    _fields_ = [
        ("n_levels", ctypes.c_int),
        ("base_n", ctypes.c_int * 3),
        ("box", ctypes.c_double),
        ("nest_n", (ctypes.c_int * 3) * (MG_MAX_LEVELS - 1)),
        ("nest_off", (ctypes.c_int * 3) * (MG_MAX_LEVELS - 1)),
        ("order", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("max_cycles", ctypes.c_int),
        ("inner_cycles", ctypes.c_int),
        ("flags", ctypes.c_int),
        ("tile_rows", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("dev_alloc", _ALLOC_FN),
        ("dev_free", _FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
    ]


class MGInfo(ctypes.Structure):
    _fields_ = [
        ("cycles", ctypes.c_int),
        ("rel_residual", ctypes.c_double),
        ("source_mean", ctypes.c_double),
        ("history", ctypes.c_double * MG_MAX_HISTORY),
        ("inner_cycles", ctypes.c_int),
        ("level_rel_residual", ctypes.c_double * MG_MAX_LEVELS),
    ]

    def as_dict(self, n_levels=MG_MAX_LEVELS):
        """The record as a dict; level_rel_residual keeps the first n_levels entries
        (the leaf levels, base first)."""
        return {"cycles": self.cycles, "rel_residual": self.rel_residual,
                "source_mean": self.source_mean, "inner_cycles": self.inner_cycles,
                "history": [self.history[i] for i in range(min(self.cycles, MG_MAX_HISTORY))],
                "level_rel_residual": [self.level_rel_residual[i] for i in range(n_levels)]}


class MGServerResult(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_longlong),
        ("status", ctypes.c_int),
        ("info1", MGInfo),
        ("info2", MGInfo),
        ("t_submit", ctypes.c_double),
        ("t_start", ctypes.c_double),
        ("t_done", ctypes.c_double),
        ("error", ctypes.c_char * 160),
    ]


class MGServerStats(ctypes.Structure):
    _fields_ = [
        ("resident_bytes", ctypes.c_ulonglong),
        ("peak_bytes", ctypes.c_ulonglong),
        ("budget_bytes", ctypes.c_ulonglong),
        ("created", ctypes.c_longlong),
        ("evictions", ctypes.c_longlong),
        ("completed", ctypes.c_longlong),
        ("pending", ctypes.c_int),
        ("active", ctypes.c_int),
        ("instances", ctypes.c_int),
        ("peak_active", ctypes.c_int),
        ("sched_cpu_s", ctypes.c_double),
        ("sched_busy_s", ctypes.c_double),
        ("uptime_s", ctypes.c_double),
        ("passes", ctypes.c_longlong),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


MG_K_FAMILIES = 9
FAMILY_NAMES = ["smooth", "restrict", "fas", "prolong", "ghost", "coarsest", "norm", "lpt", "copy"]


class MGStats(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_longlong * MG_K_FAMILIES),
        ("cells", ctypes.c_longlong * MG_K_FAMILIES),
        ("event_ms", ctypes.c_double * MG_K_FAMILIES),
        ("timed", ctypes.c_longlong * MG_K_FAMILIES),
        ("timed_cells", ctypes.c_longlong * MG_K_FAMILIES),
    ]

    def as_dict(self):
        return {name: {"launches": self.launches[i], "cells": self.cells[i],
                       "event_ms": self.event_ms[i], "timed": self.timed[i],
                       "timed_cells": self.timed_cells[i]}
                for i, name in enumerate(FAMILY_NAMES)}


class MGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS.get(status, status), message))
        self.status = status


LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libmgic.so")
_lib = None


def load_library(path=None):
    """Load libmgic.so (built by __graft_entry__.build()); raises if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise OSError("libmgic.so not found at %s; run __graft_entry__.build() first" % p)
    lib = ctypes.CDLL(p)
    vp = ctypes.c_void_p
    pp = ctypes.POINTER(ctypes.c_void_p)
    sig = {
        "mg_config_default": (None, [ctypes.POINTER(MGConfig)]),
        "mg_config_validate": (ctypes.c_int, [ctypes.POINTER(MGConfig), ctypes.c_char_p, ctypes.c_size_t]),
        "mg_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(MGConfig)]),
        "mg_total_levels": (ctypes.c_int, [ctypes.POINTER(MGConfig)]),
        "mg_hierarchy_create": (ctypes.c_int, [ctypes.POINTER(MGConfig), vp, ctypes.POINTER(vp)]),
        "mg_hierarchy_destroy": (ctypes.c_int, [vp]),
        "mg_solve_1lpt": (ctypes.c_int, [vp, pp, pp, ctypes.POINTER(MGInfo)]),
        "mg_solve_2lpt": (ctypes.c_int, [vp, pp, pp, ctypes.POINTER(MGInfo)]),
        "mg_displacements": (ctypes.c_int, [vp, pp, pp]),
        "mg_lpt2_source": (ctypes.c_int, [vp, pp, pp]),
        "mg_lpt_pipeline": (ctypes.c_int, [vp, ctypes.c_int, pp, pp, pp, pp, pp,
                                           ctypes.POINTER(MGInfo), ctypes.POINTER(MGInfo)]),
        "mg_set_stream": (ctypes.c_int, [vp, vp]),
        "mg_set_profiling": (ctypes.c_int, [vp, ctypes.c_uint]),
        "mg_set_profiling_min_cells": (ctypes.c_int, [vp, ctypes.c_longlong]),
        "mg_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(MGStats), ctypes.c_int]),
        "mg_batch_create": (ctypes.c_int, [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]),
        "mg_batch_destroy": (ctypes.c_int, [vp]),
        "mg_batch_lpt_pipeline": (ctypes.c_int, [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                 ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                                 ctypes.POINTER(MGInfo), ctypes.POINTER(MGInfo)]),
        "mg_batch_last_error": (ctypes.c_char_p, [vp]),
        "mg_last_error": (ctypes.c_char_p, [vp]),
        "mg_selftest_wait_limit": (ctypes.c_int, []),
        "mg_fp64_fma_rate": (ctypes.c_int, [ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]),
        "mg_event_pair_floor": (ctypes.c_int, [ctypes.c_int, vp, ctypes.POINTER(ctypes.c_double)]),
        "mg_selftest_persist_wait": (ctypes.c_int, []),
        "mg_batch_set_persistent_blocks": (ctypes.c_int, [vp, ctypes.c_int]),
        "mg_server_set_max_instances": (ctypes.c_int, [vp, ctypes.c_int]),
        "mg_hybrid_correction": (ctypes.c_int, [vp, vp, ctypes.POINTER(vp)]),
        "mg_lla_density": (ctypes.c_int, [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.c_double,
                                          ctypes.c_double, ctypes.POINTER(vp)]),
        "mg_white_noise": (ctypes.c_int, [ctypes.c_ulonglong, ctypes.c_longlong, vp, vp]),
        "mg_field_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                           ctypes.c_double, ctypes.POINTER(vp)]),
        "mg_field_convolve": (ctypes.c_int, [vp, vp, vp, vp]),
        "mg_field_generate": (ctypes.c_int, [vp, ctypes.c_ulonglong, vp, vp]),
        "mg_field_last_error": (ctypes.c_char_p, [vp]),
        "mg_field_destroy": (ctypes.c_int, [vp]),
        "mg_density_multiscale": (ctypes.c_int, [ctypes.POINTER(MGConfig), ctypes.c_ulonglong,
                                                 ctypes.POINTER(ctypes.c_double), ctypes.c_int,
                                                 ctypes.c_double, ctypes.POINTER(vp), vp]),
        "mg_server_create": (ctypes.c_int, [ctypes.c_ulonglong, ctypes.c_int, ctypes.POINTER(vp)]),
        "mg_server_submit": (ctypes.c_int, [vp, ctypes.c_longlong, ctypes.POINTER(MGConfig), pp, pp, pp,
                                            pp, pp]),
        "mg_server_poll": (ctypes.c_int, [vp, ctypes.POINTER(MGServerResult), ctypes.c_int,
                                          ctypes.c_double]),
        "mg_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(MGServerStats)]),
        "mg_server_destroy": (ctypes.c_int, [vp]),
        "mg_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def make_config(base_n, box, order, nests=(), precision=MG_FP64, nu1=2, nu2=2, max_cycles=50,
                tol=1e-10, inner_cycles=2, graphs=True, tile_rows=4, tma="auto", hybrid=False,
                device_loop=False, persistent=False, pair_smoother=False):
    """MGConfig from plain values; nests = [(n3, off3), ...] (off in parent cells).
    tma: smoother kernel choice, "auto" (TMA-staged tiles on float32 nests of
    >= 2^23 cells), "off" or "all"; every choice gives bit-identical results.
    hybrid: the pipelines add the hybrid Poisson correction (Sec. 3.5.2) to the
    finest level's displacements.
    device_loop: the iteration loop of every solve runs on the device (one CUDA
    graph with a while node per solve; same launches and results).
    persistent: in a Batch of mixed-precision members that all set it, the float32
    V-cycles of all members run as one persistent kernel launch per outer iteration
    (same results).
    pair_smoother: the global-memory float32 smoother updates one z-pair per thread on
    every level, instead of one z-quad per thread on levels whose rows are a multiple
    of 4 long (same results)."""
    lib = load_library()
    cfg = MGConfig()
    lib.mg_config_default(ctypes.byref(cfg))
    cfg.n_levels = 1 + len(nests)
    for a in range(3):
        cfg.base_n[a] = int(base_n[a])
    cfg.box = float(box)
    for i, (n, off) in enumerate(nests):
        for a in range(3):
            cfg.nest_n[i][a] = int(n[a])
            cfg.nest_off[i][a] = int(off[a])
    cfg.order = int(order)
    cfg.precision = int(precision)
    cfg.nu1, cfg.nu2, cfg.max_cycles, cfg.tol = int(nu1), int(nu2), int(max_cycles), float(tol)
    cfg.inner_cycles = int(inner_cycles)
    cfg.flags = (0 if graphs else MG_FLAG_NO_GRAPHS) | _TMA_FLAGS[tma] | \
        (MG_FLAG_HYBRID if hybrid else 0) | (MG_FLAG_DEVICE_LOOP if device_loop else 0) | \
        (MG_FLAG_PERSISTENT if persistent else 0) | (MG_FLAG_PAIR_SMOOTHER if pair_smoother else 0)
    cfg.tile_rows = int(tile_rows)
    return cfg


def config_from_geometry(geom, **kw):
    return make_config(geom.base_n, geom.box, geom.order, [(n.n, n.off) for n in geom.nests], **kw)


def validate(cfg):
    lib = load_library()
    buf = ctypes.create_string_buffer(512)
    st = lib.mg_config_validate(ctypes.byref(cfg), buf, 512)
    return st, buf.value.decode()


def workspace_bytes(cfg):
    return int(load_library().mg_workspace_bytes(ctypes.byref(cfg)))


def _ptrs(tensors, shapes=None, host=False):
    """Array of raw pointers; every tensor must be a contiguous float64 tensor of
    the level's shape, on the GPU (or in pinned host memory when host=True)."""
    arr = (ctypes.c_void_p * len(tensors))()
    for i, t in enumerate(tensors):
        if t is None:
            arr[i] = None
            continue
        if str(t.dtype) != "torch.float64":
            raise ValueError("tensor %d: dtype %s, expected float64" % (i, t.dtype))
        if not t.is_contiguous():
            raise ValueError("tensor %d is not contiguous" % i)
        if host:
            if t.is_cuda or not t.is_pinned():
                raise ValueError("tensor %d: host buffers must be pinned CPU tensors" % i)
        elif not t.is_cuda:
            raise ValueError("tensor %d: expected a CUDA tensor" % i)
        if shapes is not None and tuple(t.shape) != tuple(shapes[i]):
            raise ValueError("tensor %d: shape %s, expected %s" % (i, tuple(t.shape), shapes[i]))
        arr[i] = t.data_ptr()
    return arr


class Hierarchy:
    """A device-resident hierarchy (opaque C handle) bound to a CUDA stream.

    Inputs/outputs are torch float64 tensors on the GPU (or pinned CPU tensors
    for pipeline(host=True)); all arithmetic happens in libmgic.so."""

    def __init__(self, cfg, stream=None, torch_allocator=True):
        import torch
        self._torch = torch
        self.lib = load_library()
        # a private copy: the allocator fields set below belong to this hierarchy, and
        # the caller's struct may be shared by threads creating hierarchies at once
        cfg = MGConfig.from_buffer_copy(cfg)
        self.cfg = cfg
        self.shapes = [tuple(cfg.base_n)] + [tuple(cfg.nest_n[i]) for i in range(cfg.n_levels - 1)]
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep = []
        if torch_allocator:
            dev, strm = self.device.index, self.stream

            def _alloc(nbytes, ctx):
                return torch.cuda.caching_allocator_alloc(int(nbytes), dev, strm)

            def _free(ptr, ctx):
                torch.cuda.caching_allocator_delete(ptr)

            cfg.dev_alloc = _ALLOC_FN(_alloc)
            cfg.dev_free = _FREE_FN(_free)
            self._keep += [cfg.dev_alloc, cfg.dev_free]
        handle = ctypes.c_void_p()
        st = self.lib.mg_hierarchy_create(ctypes.byref(cfg), ctypes.c_void_p(self.stream.cuda_stream),
                                          ctypes.byref(handle))
        if st != 0:
            raise MGError(st, "mg_hierarchy_create: " + validate(cfg)[1])
        self.h = handle

    def _check(self, st, what, allow_noconv=False):
        if st == 0 or (allow_noconv and st == 3):
            return
        msg = self.lib.mg_last_error(self.h)
        raise MGError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def _empty(self, shape):
        return self._torch.empty(shape, dtype=self._torch.float64, device=self.device)

    def solve_1lpt(self, deltas, allow_noconv=False):
        phis = [self._empty(s) for s in self.shapes]
        info = MGInfo()
        st = self.lib.mg_solve_1lpt(self.h, _ptrs(deltas, self.shapes), _ptrs(phis), ctypes.byref(info))
        self._check(st, "mg_solve_1lpt", allow_noconv)
        return phis, info.as_dict(len(self.shapes))

    def solve_2lpt(self, phi1, allow_noconv=False):
        phis = [self._empty(s) for s in self.shapes]
        info = MGInfo()
        st = self.lib.mg_solve_2lpt(self.h, _ptrs(phi1, self.shapes), _ptrs(phis), ctypes.byref(info))
        self._check(st, "mg_solve_2lpt", allow_noconv)
        return phis, info.as_dict(len(self.shapes))

    def lpt2_source(self, phi1):
        taus = [self._empty(s) for s in self.shapes]
        st = self.lib.mg_lpt2_source(self.h, _ptrs(phi1, self.shapes), _ptrs(taus))
        self._check(st, "mg_lpt2_source")
        return taus

    def displacements(self, phi):
        disp = [[self._empty(s) for _ in range(3)] for s in self.shapes]
        flat = [d for level in disp for d in level]
        st = self.lib.mg_displacements(self.h, _ptrs(phi, self.shapes), _ptrs(flat))
        self._check(st, "mg_displacements")
        return disp

    def hybrid_correction(self, f, psi):
        """psi (3 dense tensors of the finest level) += the hybrid Poisson correction
        of the finest level's source f (mg_hybrid_correction); returns psi."""
        shape = self.shapes[-1]
        fp = _ptrs([f], [shape])
        st = self.lib.mg_hybrid_correction(self.h, ctypes.c_void_p(fp[0]), _ptrs(list(psi), [shape] * 3))
        self._check(st, "mg_hybrid_correction")
        return psi

    def lla_density(self, phi1, phi2=None, a1=1.0, a2=0.0):
        """rho / rho_bar per leaf level by the local Lagrangian approximation of the
        displacement -grad(a1 phi1 + a2 phi2) (mg_lla_density)."""
        rho = [self._empty(s) for s in self.shapes]
        st = self.lib.mg_lla_density(self.h, _ptrs(phi1, self.shapes),
                                     _ptrs(phi2, self.shapes) if phi2 is not None else None,
                                     float(a1), float(a2), _ptrs(rho))
        self._check(st, "mg_lla_density")
        return rho

    def pipeline(self, deltas, outputs=None, host=False, allow_noconv=False):
        """Whole step; `outputs` = dict of preallocated lists (phi1, phi2, disp1, disp2)."""
        if outputs is None:
            mk = (lambda s: self._torch.empty(s, dtype=self._torch.float64, pin_memory=True)) if host \
                else self._empty
            outputs = {"phi1": [mk(s) for s in self.shapes], "phi2": [mk(s) for s in self.shapes],
                       "disp1": [mk(s) for s in self.shapes for _ in range(3)],
                       "disp2": [mk(s) for s in self.shapes for _ in range(3)]}
        i1, i2 = MGInfo(), MGInfo()
        disp_shapes = [s for s in self.shapes for _ in range(3)]
        st = self.lib.mg_lpt_pipeline(self.h, 1 if host else 0, _ptrs(deltas, self.shapes, host),
                                      _ptrs(outputs["phi1"], self.shapes, host),
                                      _ptrs(outputs["phi2"], self.shapes, host),
                                      _ptrs(outputs["disp1"], disp_shapes, host),
                                      _ptrs(outputs["disp2"], disp_shapes, host),
                                      ctypes.byref(i1), ctypes.byref(i2))
        self._check(st, "mg_lpt_pipeline", allow_noconv)
        return outputs, i1.as_dict(len(self.shapes)), i2.as_dict(len(self.shapes))

    def set_stream(self, stream):
        """Order later calls against `stream` (a torch.cuda.Stream)."""
        self._check(self.lib.mg_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream)), "mg_set_stream")
        self.stream = stream

    def set_profiling(self, families=(), min_cells=0):
        """Time the launches of the named kernel families that process at least
        min_cells cells with CUDA events."""
        mask = 0
        for name in families:
            mask |= 1 << FAMILY_NAMES.index(name)
        self._check(self.lib.mg_set_profiling_min_cells(self.h, ctypes.c_longlong(int(min_cells))),
                    "mg_set_profiling_min_cells")
        self._check(self.lib.mg_set_profiling(self.h, mask), "mg_set_profiling")

    def stats(self, reset=False):
        st = MGStats()
        self._check(self.lib.mg_get_stats(self.h, ctypes.byref(st), 1 if reset else 0), "mg_get_stats")
        return st.as_dict()

    def close(self):
        if getattr(self, "h", None):
            self.lib.mg_hierarchy_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Independent hierarchies solved together: each iteration of all members
    that have not converged is one CUDA-graph launch (one branch per member)."""

    def __init__(self, hierarchies, stream=None):
        import torch
        self._torch = torch
        self.members = list(hierarchies)
        self.lib = load_library()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (ctypes.c_void_p * len(self.members))(*[m.h.value for m in self.members])
        handle = ctypes.c_void_p()
        st = self.lib.mg_batch_create(arr, len(self.members), ctypes.c_void_p(self.stream.cuda_stream),
                                      ctypes.byref(handle))
        if st != 0:
            raise MGError(st, "mg_batch_create")
        self.b = handle

    def set_persistent_blocks(self, blocks_per_sm):
        """Blocks per SM of the persistent launch of the MG_FLAG_PERSISTENT members (0:
        as many as fit)."""
        st = self.lib.mg_batch_set_persistent_blocks(self.b, int(blocks_per_sm))
        if st != 0:
            raise MGError(st, "mg_batch_set_persistent_blocks")

    def pipeline(self, deltas, outputs=None, host=False, allow_noconv=False):
        """deltas[i]: member i's per-level inputs; returns (outputs, infos1, infos2),
        outputs[i] a dict like Hierarchy.pipeline's."""
        n = len(self.members)
        if outputs is None:
            outputs = []
            for m in self.members:
                mk = (lambda s: self._torch.empty(s, dtype=self._torch.float64, pin_memory=True)) if host \
                    else m._empty
                outputs.append({"phi1": [mk(s) for s in m.shapes], "phi2": [mk(s) for s in m.shapes],
                                "disp1": [mk(s) for s in m.shapes for _ in range(3)],
                                "disp2": [mk(s) for s in m.shapes for _ in range(3)]})
        keep = []

        def table(key):
            rows = (ctypes.c_void_p * n)()
            for i, m in enumerate(self.members):
                shapes = m.shapes if key in ("delta", "phi1", "phi2") else [s for s in m.shapes for _ in range(3)]
                src = deltas[i] if key == "delta" else outputs[i][key]
                row = _ptrs(src, shapes, host)
                keep.append(row)
                rows[i] = ctypes.cast(row, ctypes.c_void_p)
            return rows

        i1 = (MGInfo * n)()
        i2 = (MGInfo * n)()
        st = self.lib.mg_batch_lpt_pipeline(self.b, 1 if host else 0, table("delta"), table("phi1"),
                                            table("phi2"), table("disp1"), table("disp2"), i1, i2)
        if not (st == 0 or (allow_noconv and st == 3)):
            msg = self.lib.mg_batch_last_error(self.b)
            raise MGError(st, "mg_batch_lpt_pipeline: " + (msg.decode() if msg else ""))
        return (outputs, [x.as_dict(len(m.shapes)) for x, m in zip(i1, self.members)],
                [x.as_dict(len(m.shapes)) for x, m in zip(i2, self.members)])

    def close(self):
        if getattr(self, "b", None):
            self.lib.mg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def selftest_wait_limit():
    """Runs the device wait-limit self-test (about 2 s); returns the status name,
    "MG_ETIMEOUT" when the bounded wait and its error path work."""
    return STATUS.get(int(load_library().mg_selftest_wait_limit()), "unknown")


def selftest_persist_wait():
    """Runs the persistent batch kernel's wait-limit self-test (about 0.1 s); returns
    the status name, "MG_ETIMEOUT" when the bounded wait and its error path work."""
    return STATUS.get(int(load_library().mg_selftest_persist_wait()), "unknown")


def fp64_fma_rate(iters=4096, stream=None):
    """FP64 fused multiply-adds per second the current device issues
    (mg_fp64_fma_rate): the measured denominator of the float64 stencils' roofline."""
    out = ctypes.c_double(0.0)
    sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    st = load_library().mg_fp64_fma_rate(int(iters), sp, ctypes.byref(out))
    if st != 0:
        raise MGError(st, "mg_fp64_fma_rate")
    return out.value


def event_pair_floor(pairs=200, stream=None):
    """Microseconds a CUDA-event pair reads around an empty kernel node of a CUDA graph
    (mg_event_pair_floor): the fixed cost inside every event-timed launch of the
    profiled kernel families."""
    out = ctypes.c_double(0.0)
    sp = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
    st = load_library().mg_event_pair_floor(int(pairs), sp, ctypes.byref(out))
    if st != 0:
        raise MGError(st, "mg_event_pair_floor")
    return out.value


def _dense_f64(t, name):
    import torch
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda \
            or not t.is_contiguous():
        raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    return ctypes.c_void_p(t.data_ptr())


def white_noise(seed, n, out=None, stream=None):
    """n standard normal deviates from Philox4x32-10 (see mg_white_noise), on the GPU."""
    import torch
    if out is None:
        out = torch.empty(int(n), dtype=torch.float64, device="cuda")
    if out.numel() != int(n):
        raise ValueError("out must hold n elements")
    stream = stream or torch.cuda.current_stream()
    st = load_library().mg_white_noise(int(seed), int(n), _dense_f64(out, "out"),
                                       ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise MGError(st, "mg_white_noise")
    return out


class Field:
    """Periodic Gaussian field generator for one grid size (mg_field_*):
    delta = IFFT[A(|k|) FFT[noise]] with A linearly interpolated from `amp`
    sampled at |k| = t dk."""

    def __init__(self, shape, h, amp, dk):
        import numpy as np
        self.lib = load_library()
        self.shape = tuple(int(n) for n in shape)
        table = np.ascontiguousarray(amp, dtype=np.float64)
        handle = ctypes.c_void_p()
        st = self.lib.mg_field_create(self.shape[0], self.shape[1], self.shape[2], float(h),
                                      table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      int(table.size), float(dk), ctypes.byref(handle))
        if st != 0:
            raise MGError(st, "mg_field_create")
        self.g = handle

    def _out(self, out):
        import torch
        if out is None:
            out = torch.empty(self.shape, dtype=torch.float64, device="cuda")
        if tuple(out.shape) != self.shape:
            raise ValueError("output shape %s != %s" % (tuple(out.shape), self.shape))
        return out

    def _check(self, st, what):
        if st != 0:
            msg = self.lib.mg_field_last_error(self.g)
            raise MGError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def convolve(self, noise, out=None, stream=None):
        import torch
        out = self._out(out)
        if tuple(noise.shape) != self.shape:
            raise ValueError("noise shape %s != %s" % (tuple(noise.shape), self.shape))
        stream = stream or torch.cuda.current_stream()
        self._check(self.lib.mg_field_convolve(self.g, _dense_f64(noise, "noise"),
                                               _dense_f64(out, "out"),
                                               ctypes.c_void_p(stream.cuda_stream)),
                    "mg_field_convolve")
        return out

    def generate(self, seed, out=None, stream=None):
        import torch
        out = self._out(out)
        stream = stream or torch.cuda.current_stream()
        self._check(self.lib.mg_field_generate(self.g, int(seed), _dense_f64(out, "out"),
                                               ctypes.c_void_p(stream.cuda_stream)),
                    "mg_field_generate")
        return out

    def close(self):
        if getattr(self, "g", None):
            self.lib.mg_field_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def density_multiscale(cfg, seed, sqrt_p, dk, out=None, stream=None):
    """delta on every leaf level of the hierarchy cfg describes (mg_density_multiscale);
    sqrt_p: sqrt(P(|k|)) sampled at |k| = t dk.  Returns the list of device tensors."""
    import numpy as np
    import torch
    shapes = [tuple(cfg.base_n)] + [tuple(cfg.nest_n[i]) for i in range(cfg.n_levels - 1)]
    if out is None:
        out = [torch.empty(sh, dtype=torch.float64, device="cuda") for sh in shapes]
    table = np.ascontiguousarray(sqrt_p, dtype=np.float64)
    stream = stream or torch.cuda.current_stream()
    st = load_library().mg_density_multiscale(
        ctypes.byref(cfg), int(seed), table.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
        int(table.size), float(dk), _ptrs(out, shapes), ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise MGError(st, "mg_density_multiscale")
    return out
