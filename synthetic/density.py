"""Multi-scale Gaussian source field delta on every level of a hierarchy.

Follows the structure of Sec. 2.1-2.3 of Hahn & Abel 2011 in simplified form:

* white noise mu ~ N(0, 1) per cell, numpy PCG64, C order; nest noise is made
  consistent with its parent by the Hoffman-Ribak constraint (Sec. 2.3.1):
  the mean of the 8 children of a parent cell is replaced by the parent value
  (scaled by 1/sqrt(8) for unit-variance cells);
* the base level is a periodic FFT convolution of the noise with the
  k-space-sampled amplitude sqrt(P(k)/h^3) (eq. of Sec. 2.1);
* a nest gets delta_self, an isolated convolution of its own noise on a grid
  zero-padded to twice its size (Sec. 2.3.3, item 2), plus delta_coarse, the
  parent-level field due to all noise outside the nest, carried down the
  chain with conservative tricubic interpolation (Sec. 2.3.3 item 1; 2.3.4);
* covered parent cells finally hold the average of their 8 children.

The boundary term delta_bnd and the real-space (FFTlog) kernel are left out:
these inputs only have to look like the paper's fields (Gaussian, the stated
spectrum, continuous across coarse-fine boundaries); the solver sees them as
given data.
"""

from typing import List

import numpy as np

from .geometry import Geometry
from .spectra import BBKSPower, PowerLaw


def white_noise(shape, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal(tuple(shape))


def _kmag(shape, h):
    axes = [2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in shape]
    kx, ky, kz = np.meshgrid(*axes, indexing="ij")
    return np.sqrt(kx * kx + ky * ky + kz * kz)


def _convolve_periodic(noise, h, power):
    amp = np.sqrt(power(_kmag(noise.shape, h)) / h ** 3)
    return np.ascontiguousarray(np.fft.ifftn(np.fft.fftn(noise) * amp).real)


def _convolve_isolated(noise, h, power):
    shape = noise.shape
    padded = np.zeros(tuple(2 * n for n in shape))
    padded[:shape[0], :shape[1], :shape[2]] = noise
    out = _convolve_periodic(padded, h, power)
    return np.ascontiguousarray(out[:shape[0], :shape[1], :shape[2]])


def _children_mean(a):
    n = a.shape
    return a.reshape(n[0] // 2, 2, n[1] // 2, 2, n[2] // 2, 2).mean(axis=(1, 3, 5))


def _inject(c):
    return np.repeat(np.repeat(np.repeat(c, 2, axis=0), 2, axis=1), 2, axis=2)


def _cubic_weights(t):
    """Lagrange weights through nodes -1, 0, 1, 2 evaluated at t."""
    return np.array([-t * (t - 1) * (t - 2) / 6.0,
                     (t + 1) * (t - 1) * (t - 2) / 2.0,
                     -(t + 1) * t * (t - 2) / 2.0,
                     (t + 1) * t * (t - 1) / 6.0])


def _tricubic_conservative(parent, off, n):
    """Interpolate a parent-level field onto the nest of size n at offset off.

    Each fine cell centre sits at -1/4 or +1/4 parent cells from its parent's
    centre; tensor cubic Lagrange interpolation through 4 parent cells, then
    each group of 8 children is shifted to average to the parent value."""
    out = parent
    for axis in range(3):
        nf = n[axis]
        idx = np.arange(nf)
        p = off[axis] + idx // 2
        # Fine centre in parent-index units: p - 1/4 (even i) or p + 1/4 (odd i).
        # Nodes base..base+3 are local coordinates -1, 0, 1, 2.
        odd = idx % 2 == 1
        base = np.where(odd, p - 1, p - 2)
        t = np.where(odd, 0.25, 0.75)
        w = _cubic_weights(t)  # shape (4, nf)
        moved = np.moveaxis(out, axis, 0)
        acc = np.zeros((nf,) + moved.shape[1:])
        for s in range(4):
            acc += w[s].reshape((nf,) + (1,) * (moved.ndim - 1)) * moved[base + s]
        out = np.moveaxis(acc, 0, axis)
    # out now has the fine extent along every axis
    sl = tuple(slice(off[a], off[a] + n[a] // 2) for a in range(3))
    coarse = parent[sl]
    return out + _inject(coarse - _children_mean(out))


def make_delta(geom: Geometry, seed: int, power=None) -> List[np.ndarray]:
    """delta on every level (base first), float64, C-ordered [x][y][z]."""
    if power is None:
        power = BBKSPower()
    h = geom.box / geom.base_n[0]
    noise = white_noise(geom.base_n, seed)
    deltas = [_convolve_periodic(noise, h, power)]

    def region(nest):
        return tuple(slice(nest.off[a], nest.off[a] + nest.n[a] // 2) for a in range(3))

    def outside_field(mu, h_l, periodic, child):
        masked = mu.copy()
        masked[region(child)] = 0.0
        conv = _convolve_periodic if periodic else _convolve_isolated
        return conv(masked, h_l, power)

    ext = outside_field(noise, h, True, geom.nests[0]) if geom.nests else None
    mu_parent = noise
    for lvl, nest in enumerate(geom.nests, start=1):
        h = h / 2.0
        mu = white_noise(nest.n, seed * 1000 + lvl)
        coarse_noise = mu_parent[region(nest)] / np.sqrt(8.0)
        mu = mu - _inject(_children_mean(mu)) + _inject(coarse_noise)
        carried = _tricubic_conservative(ext, nest.off, nest.n)
        deltas.append(_convolve_isolated(mu, h, power) + carried)
        if lvl < len(geom.nests):
            ext = outside_field(mu, h, False, geom.nests[lvl]) + carried
        mu_parent = mu
    for lvl in range(len(geom.nests), 0, -1):
        deltas[lvl - 1][region(geom.nests[lvl - 1])] = _children_mean(deltas[lvl])
    return deltas


def make_delta_powerlaw(shape, seed: int, index: float = -2.0, box: float = 1.0) -> np.ndarray:
    """Single periodic level: noise convolved with P(k) ∝ k^index, rescaled to unit RMS."""
    delta = _convolve_periodic(white_noise(shape, seed), box / shape[0], PowerLaw(index))
    return delta / np.sqrt(np.mean(delta * delta))
