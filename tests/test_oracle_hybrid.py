"""Pins of the hybrid-correction oracle (Sec. 3.5.2): on a periodic level the
finite-difference displacement plus the correction is the exact continuum
spectral displacement of the source; on a zero-padded nest it is the same
statement on the padded periodic box, restricted to the nest; the correction is
small for smooth sources and shrinks with the stencil order."""

import numpy as np
import pytest

from oracle.fft_solve import exact_solve
from oracle.hierarchy import Hierarchy
from oracle.hybrid import hybrid_correction
from oracle.lpt import gradient
from synthetic import Geometry


def _continuum_psi(f, h):
    """psi = -grad phi with lap phi = f, exactly in k space (zero mode removed)."""
    fk = np.fft.fftn(f)
    k = np.meshgrid(*[2 * np.pi * np.fft.fftfreq(n, d=h) for n in f.shape], indexing="ij")
    ksq = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    ksq.flat[0] = 1.0
    out = []
    for j in range(3):
        m = 1j * k[j] / ksq
        m.flat[0] = 0.0
        out.append(np.fft.ifftn(m * fk).real)
    return out


def _fd_psi(f, h, order):
    """Finite-difference psi = -G phi of the periodic finite-difference solution."""
    phi = exact_solve(f - f.mean(), h, order)
    geom = Geometry(f.shape, h * f.shape[0], order, ())
    return gradient(Hierarchy(geom), [phi])[0]


@pytest.mark.parametrize("order", (2, 4, 6))
@pytest.mark.parametrize("shape", [(16, 16, 16), (12, 10, 14), (9, 11, 8)])
def test_periodic_level_becomes_exact(order, shape):
    rng = np.random.Generator(np.random.PCG64(order))
    f = rng.standard_normal(shape)
    h = 0.5
    fd = _fd_psi(f, h, order)
    corr = hybrid_correction(f, h, order, pad=False)
    ex = _continuum_psi(f, h)
    for a in range(3):
        np.testing.assert_allclose(fd[a] + corr[a], ex[a], atol=1e-11 * np.abs(ex[a]).max())


@pytest.mark.parametrize("order", (2, 6))
def test_padded_nest_is_exact_on_the_padded_box(order):
    n, h = 12, 0.25
    rng = np.random.Generator(np.random.PCG64(9))
    f = rng.standard_normal((n, n, n))
    padded = np.zeros((2 * n,) * 3)
    padded[:n, :n, :n] = f
    fd = _fd_psi(padded, h, order)
    ex = _continuum_psi(padded, h)
    corr = hybrid_correction(f, h, order, pad=True)
    for a in range(3):
        want = (ex[a] - fd[a])[:n, :n, :n]
        np.testing.assert_allclose(corr[a], want, atol=1e-11 * np.abs(want).max())


def test_correction_is_small_for_smooth_sources_and_shrinks_with_order():
    n, h = 32, 1.0
    x = np.arange(n) - n / 2 + 0.5
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    f = np.exp(-(X ** 2 + Y ** 2 + Z ** 2) / (2 * 4.0 ** 2))
    rel = []
    for order in (2, 4, 6):
        corr = hybrid_correction(f, h, order, pad=True)
        padded = np.zeros((2 * n,) * 3)
        padded[:n, :n, :n] = f
        psi = _continuum_psi(padded, h)[0][:n, :n, :n]
        rel.append(np.abs(corr[0]).max() / np.abs(psi).max())
    assert rel[0] < 0.05 and rel[0] > rel[1] > rel[2] > 0.0
