"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Tolerance (float64 path): <= 1e-10 RMS relative error in phi and in the
displacements.  At a matched V-cycle count both sides run the same
algorithm, so the expected difference is rounding (~1e-14); converged runs
are compared against the exact DFT solve and the oracle's converged solve.
"""

import numpy as np
import pytest

from oracle.fft_solve import exact_solve, spectral_gradient
from oracle.lpt import gradient as oracle_gradient
from oracle.lpt import lpt2_source as oracle_tau
from oracle.lpt import lpt_pipeline
from oracle.hierarchy import Hierarchy as OracleHierarchy
from oracle.hierarchy import restrict
from oracle.multigrid import solve as oracle_solve
from synthetic import (Geometry, NestSpec, config_zoom2, make_delta, make_delta_powerlaw,
                       small_zoom)

pytestmark = pytest.mark.gpu
TOL = 1e-10


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1103_6031_gb300 as pkg
    return pkg


def rel(a, b):
    a = a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)
    b = np.asarray(b)
    return float(np.sqrt(np.sum((a - b) ** 2) / max(np.sum(b * b), 1e-300)))


def to_dev(arrs):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in arrs]


def hier(lib, geom, **kw):
    return lib.Hierarchy(lib.config_from_geometry(geom, **kw))


def test_unigrid64_order2_matches_oracle_and_dft(lib):
    d = make_delta_powerlaw((64,) * 3, 1)
    geom = Geometry((64,) * 3, 1.0, 2, ())
    h = hier(lib, geom, tol=1e-10)
    phis, info = h.solve_1lpt(to_dev([d]))
    ref, rinfo = oracle_solve(geom, [d], tol=1e-10)
    assert info["cycles"] == rinfo["cycles"]
    assert info["rel_residual"] <= 1e-10
    assert rel(phis[0], ref[0]) < TOL
    np.testing.assert_allclose(info["history"], rinfo["history"], rtol=1e-6, atol=1e-14)
    disp = h.displacements(phis)
    psi = oracle_gradient(OracleHierarchy(geom), ref)
    for a in range(3):
        assert rel(disp[0][a], psi[0][a]) < TOL
    # converged tightly, the result is the exact DFT solve of the same operator
    h2 = hier(lib, geom, tol=1e-13)
    phis2, _ = h2.solve_1lpt(to_dev([d]))
    ex = exact_solve(d - d.mean(), 1.0 / 64, 2)
    assert rel(phis2[0], ex) < TOL
    gex = spectral_gradient(ex, 1.0 / 64, 2)
    disp2 = h2.displacements(phis2)
    for a in range(3):
        assert rel(disp2[0][a], gex[a]) < TOL


GEOMS = [
    small_zoom(16, ((16, 4),), order=2, box=50.0),
    small_zoom(24, ((20, 7), (16, 6)), order=4, box=50.0),
    small_zoom(24, ((12, 6),), order=6, box=50.0),
    small_zoom(32, ((24, 8), (20, 6)), order=6, box=80.0),
]


@pytest.mark.parametrize("geom", GEOMS, ids=lambda g: "o%d_L%d" % (g.order, g.n_levels))
def test_nested_pipeline_matched_cycles(lib, geom):
    deltas = make_delta(geom, 21)
    cycles = 3
    ref = lpt_pipeline(geom, deltas, tol=0.0, cycles=cycles)
    h = hier(lib, geom, tol=0.0, max_cycles=cycles)
    out, i1, i2 = h.pipeline(to_dev(deltas))
    assert i1["cycles"] == cycles and i2["cycles"] == cycles
    np.testing.assert_allclose(i1["history"], ref["info1"]["history"], rtol=1e-6, atol=1e-14)
    np.testing.assert_allclose(i2["history"], ref["info2"]["history"], rtol=1e-6, atol=1e-14)
    # per-level relative residuals of the last cycle (Sec. 3.2 norm, level by level)
    np.testing.assert_allclose(i1["level_rel_residual"], ref["info1"]["level_rel_residual"],
                               rtol=1e-6, atol=1e-14)
    np.testing.assert_allclose(i2["level_rel_residual"], ref["info2"]["level_rel_residual"],
                               rtol=1e-6, atol=1e-14)
    for l in range(geom.n_levels):
        assert rel(out["phi1"][l], ref["phi1"][l]) < TOL
        assert rel(out["phi2"][l], ref["phi2"][l]) < TOL
        for a in range(3):
            assert rel(out["disp1"][3 * l + a], ref["psi1"][l][a]) < TOL
            assert rel(out["disp2"][3 * l + a], ref["psi2"][l][a]) < TOL


@pytest.mark.parametrize("geom", GEOMS[1:3], ids=lambda g: "o%d_L%d" % (g.order, g.n_levels))
def test_lpt2_source_matches(lib, geom):
    rng = np.random.default_rng(5)
    phis = [rng.standard_normal(n) for n in [geom.base_n] + [x.n for x in geom.nests]]
    taus = oracle_tau(OracleHierarchy(geom), phis)
    for l in range(len(taus) - 1, 0, -1):
        r = OracleHierarchy(geom).covered_region(OracleHierarchy(geom).base + l)
        taus[l - 1][r] = restrict(taus[l])
    h = hier(lib, geom)
    got = h.lpt2_source(to_dev(phis))
    for l in range(len(taus)):
        assert rel(got[l], taus[l]) < TOL


@pytest.mark.parametrize("order", (2, 4, 6))
def test_converged_nested_matches_converged_oracle(lib, order):
    geom = small_zoom(24, ((20, 7),), order=order, box=30.0)
    deltas = make_delta(geom, 8)
    ref, rinfo = oracle_solve(geom, deltas, tol=1e-12)
    h = hier(lib, geom, tol=1e-12)
    phis, info = h.solve_1lpt(to_dev(deltas))
    assert info["rel_residual"] <= 1e-12
    hist = info["history"]
    assert all(a / b >= 10.0 for a, b in zip(hist[:-1], hist[1:])), hist
    for l in range(geom.n_levels):
        assert rel(phis[l], ref[l]) < TOL


def test_host_buffers_equal_device_buffers(lib):
    import torch
    geom = GEOMS[1]
    deltas = make_delta(geom, 4)
    h = hier(lib, geom, tol=1e-11)
    dev, _, _ = h.pipeline(to_dev(deltas))
    host_in = [torch.from_numpy(x).pin_memory() for x in deltas]
    host, _, _ = h.pipeline(host_in, host=True)
    for key in ("phi1", "phi2", "disp1", "disp2"):
        for a, b in zip(dev[key], host[key]):
            assert torch.equal(a.cpu(), b)


@pytest.mark.parametrize("geom", [
    Geometry((48, 48, 48), 10.0, 6, ()),
    Geometry((24, 32, 40), 24.0, 6, (NestSpec((14, 20, 18), (7, 6, 9)),)),
    Geometry((34, 34, 34), 1.0, 2, (NestSpec((18, 18, 18), (9, 8, 11)),)),
], ids=["base48", "aniso", "base34"])
def test_ragged_geometries_match(lib, geom):
    deltas = make_delta(geom, 13)
    ref, rinfo = oracle_solve(geom, deltas, tol=0.0, cycles=3)
    h = hier(lib, geom, tol=0.0, max_cycles=3)
    phis, info = h.solve_1lpt(to_dev(deltas))
    for l in range(geom.n_levels):
        assert rel(phis[l], ref[l]) < TOL


def test_zoom2_full_size(lib):
    geom = config_zoom2()
    deltas = make_delta(geom, 2)
    ref, rinfo = oracle_solve(geom, deltas, tol=0.0, cycles=2)
    h = hier(lib, geom, tol=0.0, max_cycles=2)
    phis, info = h.solve_1lpt(to_dev(deltas))
    for l in range(2):
        assert rel(phis[l], ref[l]) < TOL
    np.testing.assert_allclose(info["history"], rinfo["history"], rtol=1e-6, atol=1e-14)
    h2 = hier(lib, geom, tol=1e-10)
    phis, info = h2.solve_1lpt(to_dev(deltas))
    hist = info["history"]
    assert info["rel_residual"] <= 1e-10
    assert all(a / b >= 10.0 for a, b in zip(hist[:-1], hist[1:])), hist


def test_errors_are_reported(lib):
    import torch
    bad = lib.make_config((32, 32, 32), 1.0, 3)
    with pytest.raises(lib.MGError) as e:
        lib.Hierarchy(bad)
    assert e.value.status == 1
    geom = GEOMS[0]
    h = hier(lib, geom, tol=1e-14, max_cycles=1)
    deltas = to_dev(make_delta(geom, 3))
    with pytest.raises(lib.MGError) as e:
        h.solve_1lpt(deltas)
    assert e.value.status == 3  # MG_ENOCONV
    phis, info = h.solve_1lpt(deltas, allow_noconv=True)
    assert info["cycles"] == 1 and np.isfinite(phis[0].cpu().numpy()).all()
    st = h.lib.mg_solve_1lpt(h.h, None, None, None)
    assert st == 1


@pytest.mark.parametrize("order", (2, 4, 6))
def test_mixed_precision_matches_fp64_oracle(lib, order):
    """MG_MIXED (float32 V-cycles inside float64 iterative refinement) reaches the
    float64 oracle's converged solution to <= 1e-6 RMS relative error in phi1, phi2
    and both displacement fields."""
    geom = small_zoom(24, ((20, 7), (16, 6)), order=order, box=50.0)
    deltas = make_delta(geom, 31)
    ref = lpt_pipeline(geom, deltas, tol=1e-12, max_cycles=40)
    h = hier(lib, geom, tol=1e-10, precision=lib.MG_MIXED, inner_cycles=2)
    out, i1, i2 = h.pipeline(to_dev(deltas))
    assert i1["rel_residual"] <= 1e-10 and i2["rel_residual"] <= 1e-10
    # first outer iteration: inner_cycles float32 V-cycles; later ones 1..inner_cycles
    assert 2 + (i1["cycles"] - 1) <= i1["inner_cycles"] <= 2 * i1["cycles"]
    for l in range(geom.n_levels):
        assert rel(out["phi1"][l], ref["phi1"][l]) <= 1e-6
        assert rel(out["phi2"][l], ref["phi2"][l]) <= 1e-6
        for a in range(3):
            assert rel(out["disp1"][3 * l + a], ref["psi1"][l][a]) <= 1e-6
            assert rel(out["disp2"][3 * l + a], ref["psi2"][l][a]) <= 1e-6


def test_deep_zoom_full_size(lib):
    """128^3 base + 4 nests of 128^3 (jittered offsets): float64 matches the oracle
    element by element at a matched cycle count, and converges at >= 10x per cycle
    down to the rounding floor (the mixed-precision step against the converged oracle
    is in test_gpu_full_size_oracle.py)."""
    from synthetic import config_deep_zoom
    geom = config_deep_zoom()
    deltas = make_delta(geom, 3)
    ref, rinfo = oracle_solve(geom, deltas, tol=0.0, cycles=2)
    h = hier(lib, geom, tol=0.0, max_cycles=2)
    phis, info = h.solve_1lpt(to_dev(deltas))
    for l in range(geom.n_levels):
        assert rel(phis[l], ref[l]) < TOL
    np.testing.assert_allclose(info["history"], rinfo["history"], rtol=1e-6, atol=1e-14)
    h.close()
    d = to_dev(deltas)
    tight = hier(lib, geom, tol=1e-12)
    b, t1, t2 = tight.pipeline(d)
    hist = t1["history"]
    # >= 10x per cycle until the float64 rounding floor of the composite residual
    assert all(x / y >= 10.0 for x, y in zip(hist[:-1], hist[1:]) if y > 1e-10), hist


@pytest.mark.parametrize("mixed", [False, True], ids=["fp64", "mixed"])
def test_zero_and_constant_sources(lib, mixed):
    """Degenerate sources: zero, and a constant (which the composite mean removal
    makes zero up to rounding): the first solve stops after one cycle at the
    rounding-level floor with phi ~ 0; tau ~ 0; no NaN anywhere, status OK."""
    import torch
    geom = small_zoom(24, ((20, 7),), order=6, box=50.0)
    kw = dict(tol=1e-10)
    if mixed:
        kw.update(precision=lib.MG_MIXED, inner_cycles=2)
    h = hier(lib, geom, **kw)
    shapes = h.shapes
    for value in (0.0, 3.5):
        d = [torch.full(s, value, dtype=torch.float64, device="cuda") for s in shapes]
        out, i1, i2 = h.pipeline(d)
        assert i1["cycles"] == 1
        for key in ("phi1", "phi2", "disp1", "disp2"):
            for x in out[key]:
                assert torch.isfinite(x).all() and x.abs().max().item() < 1e-12, key
        assert abs(i1["source_mean"] - value) < 1e-12
