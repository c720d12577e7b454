"""The C-ABI library: loads, exports every symbol of include/mg.h, and its
host-only calls (defaults, validation, workspace size, level count) behave.
No GPU is touched here."""

import ctypes
import os
import re

import pytest

from oracle.hierarchy import Hierarchy as OracleHierarchy
from synthetic import Geometry, config_batch, config_deep_zoom, config_zoom2, small_zoom


@pytest.fixture(scope="module")
def mg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300.mg as mgmod
    return mgmod


def _declared_symbols(repo_root):
    text = open(os.path.join(repo_root, "include", "mg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


def test_library_exports_every_declared_symbol(mg, repo_root):
    lib = mg.load_library()
    names = _declared_symbols(repo_root)
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    assert b"sm_103a" in lib.mg_version()


def test_default_config_is_valid(mg):
    cfg = mg.MGConfig()
    mg.load_library().mg_config_default(ctypes.byref(cfg))
    assert (cfg.order, cfg.nu1, cfg.nu2, cfg.max_cycles, cfg.tol) == (2, 2, 2, 50, 1e-10)
    assert mg.validate(cfg)[0] == 0


@pytest.mark.parametrize("bad,needle", [
    (dict(order=3), "order"),
    (dict(nests=[((15, 16, 16), (8, 8, 8))]), "even"),
    (dict(nests=[((16, 16, 16), (1, 8, 8))]), "margin"),
    (dict(nests=[((16, 16, 16), (8, 8, 23))]), "margin"),
    (dict(box=-1.0), "box"),
    (dict(max_cycles=0), "max_cycles"),
    (dict(nu1=0, nu2=0), "nu1"),
])
def test_invalid_configs_are_rejected(mg, bad, needle):
    kw = dict(base_n=(32, 32, 32), box=1.0, order=2, nests=[])
    kw.update(bad)
    cfg = mg.make_config(**kw)
    st, msg = mg.validate(cfg)
    assert st == 1 and needle in msg, msg
    assert mg.workspace_bytes(cfg) == 0


def test_allocator_callbacks_must_come_in_pairs(mg):
    cfg = mg.make_config((16, 16, 16), 1.0, 2)
    cfg.dev_alloc = mg._ALLOC_FN(lambda n, c: 0)
    st, msg = mg.validate(cfg)
    assert st == 1 and "dev_alloc" in msg


@pytest.mark.parametrize("geom", [
    Geometry((64, 64, 64), 1.0, 2, ()),
    Geometry((48, 48, 48), 1.0, 6, ()),
    Geometry((24, 32, 40), 1.0, 6, ()),
    Geometry((64, 8, 8), 1.0, 6, ()),
    small_zoom(32, ((32, 8), (20, 7)), order=4),
    config_zoom2(),
    config_deep_zoom(),
])
def test_level_chain_matches_oracle(mg, geom):
    cfg = mg.config_from_geometry(geom)
    assert mg.validate(cfg)[0] == 0
    lib = mg.load_library()
    assert lib.mg_total_levels(ctypes.byref(cfg)) == len(OracleHierarchy(geom).levels)


def test_workspace_grows_with_nests(mg):
    one = mg.workspace_bytes(mg.config_from_geometry(config_zoom2()))
    base = mg.workspace_bytes(mg.make_config((128,) * 3, 100.0, 6))
    deep = mg.workspace_bytes(mg.config_from_geometry(config_deep_zoom()))
    assert 0 < base < one < deep
    # per 128^3 leaf level: float64 u (x2), f_fas and f on the padded grid, and four dense
    # arrays staging the first solve's host outputs; plus three dense scratch arrays and
    # three padded 2LPT work arrays of one level, and the (smaller) coarsenings below the base
    padded = 136 * 134 * 134
    per_level = 4 * 8 * padded + 4 * 8 * 128 ** 3
    assert deep < (5 * per_level + 3 * 8 * 128 ** 3 + 3 * 8 * padded) * 1.1


def test_batch_geometries_are_all_valid(mg):
    for geom in config_batch():
        cfg = mg.config_from_geometry(geom)
        st, msg = mg.validate(cfg)
        assert st == 0, (geom, msg)


def test_null_handles_and_bad_arguments_are_rejected_without_a_gpu(mg):
    """Argument checks that run before any CUDA call: NULL handles and impossible
    sizes give MG_EINVAL (or -1 from mg_server_poll), destroy calls are NULL-safe."""
    lib = mg.load_library()
    out = ctypes.c_void_p()
    assert lib.mg_server_create(0, 4, ctypes.byref(out)) == 1          # no budget
    assert lib.mg_server_create(1 << 30, 0, ctypes.byref(out)) == 1    # no request slot
    assert lib.mg_server_create(1 << 30, 257, ctypes.byref(out)) == 1  # too many
    assert lib.mg_server_create(1 << 30, 4, None) == 1
    cfg = mg.make_config((32, 32, 32), 1.0, 2)
    assert lib.mg_server_submit(None, 0, ctypes.byref(cfg), None, None, None, None, None) == 1
    assert lib.mg_server_poll(None, None, 1, 0.0) == -1
    assert lib.mg_server_get_stats(None, None) == 1
    assert lib.mg_server_destroy(None) == 0
    assert lib.mg_hierarchy_destroy(None) == 0
    assert lib.mg_batch_destroy(None) == 0
    assert lib.mg_batch_create(None, 0, None, ctypes.byref(out)) == 1
    assert lib.mg_hierarchy_create(None, None, ctypes.byref(out)) == 1
    assert lib.mg_last_error(None) in (b"", None)


def test_server_cap_and_probes_reject_bad_arguments_without_a_gpu(mg):
    """mg_server_set_max_instances, mg_fp64_fma_rate and mg_event_pair_floor check their
    arguments before any CUDA call."""
    lib = mg.load_library()
    assert lib.mg_server_set_max_instances(None, 3) == 1
    out = ctypes.c_double(-1.0)
    assert lib.mg_event_pair_floor(0, None, ctypes.byref(out)) == 1
    assert lib.mg_event_pair_floor(1025, None, ctypes.byref(out)) == 1
    assert lib.mg_event_pair_floor(8, None, None) == 1
    assert lib.mg_fp64_fma_rate(8, None, ctypes.byref(out)) == 1
    assert lib.mg_fp64_fma_rate(1 << 23, None, ctypes.byref(out)) == 1
