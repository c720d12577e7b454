"""Pins of the multi-scale density oracle (Sec. 2.3): a single level reduces to
the periodic field of Sec. 2.1; the Hoffman-Ribak constraint holds exactly and
keeps unit variance; the conservative tricubic interpolation conserves the parent
values and reproduces linear fields; covered cells hold children means; the
nest's field has the statistics of a field of its resolution."""

import numpy as np

from oracle.density import (children_mean, level_noise, multiscale, tricubic_conservative)
from oracle.noise import gaussian_field, white_noise
from synthetic import Geometry, NestSpec, small_zoom
from synthetic.spectra import BBKSPower

DK = 0.01


def _table(nt=4000):
    k = np.arange(nt) * DK
    t = np.sqrt(BBKSPower()(np.maximum(k, 1e-12)))
    t[0] = 0.0
    return t


def test_single_level_is_the_periodic_field():
    geom = Geometry((16, 12, 20), 40.0, 6, ())
    h = 40.0 / 16
    table = _table()
    d = multiscale(geom, 3, table, DK)[0]
    ref = gaussian_field(white_noise(3, 16 * 12 * 20).reshape(16, 12, 20), h, table / h ** 1.5, DK)
    np.testing.assert_allclose(d, ref, rtol=0, atol=1e-14 * np.abs(ref).max())


def test_hoffman_ribak_constraint_and_variance():
    geom = small_zoom(32, ((32, 8), (32, 8)), order=6, box=50.0)
    mu = level_noise(geom, 11)
    for l, nest in enumerate(geom.nests, start=1):
        sl = tuple(slice(nest.off[a], nest.off[a] + nest.n[a] // 2) for a in range(3))
        np.testing.assert_allclose(children_mean(mu[l]), mu[l - 1][sl] / np.sqrt(8.0), atol=1e-14)
        assert abs(mu[l].var() - 1.0) < 0.05
    # the nest noise is not the parent's: its within-parent fluctuations are fresh
    assert abs(np.corrcoef(mu[1].ravel(), mu[2].ravel()[:mu[1].size])[0, 1]) < 0.05


def test_tricubic_conservative_interpolation():
    rng = np.random.Generator(np.random.PCG64(2))
    parent = rng.standard_normal((12, 14, 16))
    off, n = (3, 4, 5), (10, 8, 12)
    fine = tricubic_conservative(parent, off, n)
    sl = tuple(slice(off[a], off[a] + n[a] // 2) for a in range(3))
    np.testing.assert_allclose(children_mean(fine), parent[sl], atol=1e-13)
    # a linear field (cell centres) is reproduced exactly at the fine cell centres
    i, j, k = np.meshgrid(*[np.arange(m) for m in parent.shape], indexing="ij")
    lin = 0.3 * i - 0.7 * j + 1.1 * k + 2.0
    fine = tricubic_conservative(lin, off, n)
    fi, fj, fk = np.meshgrid(*[off[a] + (np.arange(n[a]) + 0.5) / 2.0 - 0.5 for a in range(3)],
                             indexing="ij")
    np.testing.assert_allclose(fine, 0.3 * fi - 0.7 * fj + 1.1 * fk + 2.0, atol=1e-12)


def test_covered_cells_and_nest_statistics():
    geom = Geometry((32, 32, 32), 64.0, 6, (NestSpec((32, 32, 32), (8, 8, 8)),))
    table = _table()
    d = multiscale(geom, 5, table, DK)
    sl = tuple(slice(8, 24) for _ in range(3))
    np.testing.assert_allclose(d[0][sl], children_mean(d[1]), atol=1e-14)
    # the nest field has about the variance of a periodic field of the nest's
    # resolution (the same spectrum, more small-scale power than the base)
    ref = [gaussian_field(white_noise(s, 64 ** 3).reshape((64,) * 3), 1.0, table / 1.0, DK)
           for s in (1, 2)]
    var_ref = np.mean([r.var() for r in ref])
    inner = d[1][4:28, 4:28, 4:28]
    assert 0.7 < inner.var() / var_ref < 1.3
    assert d[1].var() > d[0].var()


def test_nest_carries_the_parent_large_scales():
    """The nest's field averaged over the nest equals, up to the sub-parent-cell
    scales, the average of the parent's own periodic field over the covered cells:
    the long waves from the noise outside the nest enter through the parent's
    convolution (Sec. 2.3).  Over 16 seeds the region means agree to a few percent;
    the nest's own isolated convolution alone misses them by ~40%."""
    geom = Geometry((32, 32, 32), 64.0, 6, (NestSpec((32, 32, 32), (8, 8, 8)),))
    table = _table()
    sl = tuple(slice(8, 24) for _ in range(3))
    nest_means, parent_means = [], []
    for seed in range(16):
        d = multiscale(geom, seed, table, DK)
        mu = level_noise(geom, seed)
        parent = gaussian_field(mu[0], 2.0, table / 2.0 ** 1.5, DK)
        nest_means.append(d[1].mean())
        parent_means.append(parent[sl].mean())
    nm, pm = np.array(nest_means), np.array(parent_means)
    assert np.sqrt(np.mean((nm - pm) ** 2) / np.mean(pm ** 2)) < 0.15
