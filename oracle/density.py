"""Multi-scale density field on a nested hierarchy (Sec. 2.3), oracle of the GPU
generator (test infrastructure only: imported by tests/; nothing in the library
path imports it).

Following Sec. 2.3 in the simplified form the library implements:
* noise: level l draws Philox4x32-10 normal deviates with stream (counter word 2)
  l from the same seed (oracle/noise.py);
* a nest's noise is constrained to its parent by Hoffman-Ribak (Sec. 2.3.1): the
  mean of the 8 children of a parent cell is replaced by the parent value / sqrt(8)
  (unit-variance cells);
* the base level is the periodic convolution IFFT[A(|k|) FFT[noise]] with
  A = sqrt(P(k)) / h^{3/2} (Sec. 2.1), the amplitude table holding sqrt(P) at
  |k| = t dk;
* a nest gets delta_self, the isolated convolution of its own noise (zero-padded to
  twice its size, Sec. 2.3.3 item 2), plus delta_coarse: the parent-level field of
  all noise outside the nest (the parent's noise with the nest region zeroed,
  convolved periodically on the base, isolated on nests, plus what that level itself
  carried), brought down by conservative tricubic interpolation (Sec. 2.3.3 item 1,
  2.3.4): tensor cubic Lagrange interpolation through the 4 nearest parent cells
  (fine centres at -1/4 and +1/4 parent cells), then each group of 8 children
  shifted so that it averages to its parent value;
* covered parent cells finally hold the mean of their 8 children.
"""

import numpy as np

from .noise import amplitude, kmag, white_noise


def children_mean(a):
    n = a.shape
    return a.reshape(n[0] // 2, 2, n[1] // 2, 2, n[2] // 2, 2).mean(axis=(1, 3, 5))


def inject(c):
    return np.repeat(np.repeat(np.repeat(c, 2, axis=0), 2, axis=1), 2, axis=2)


def convolve_periodic(noise, h, sqrt_p, dk):
    a = amplitude(kmag(noise.shape, h), sqrt_p, dk) / h ** 1.5
    a.flat[0] = 0.0
    return np.ascontiguousarray(np.fft.ifftn(np.fft.fftn(noise) * a).real)


def convolve_isolated(noise, h, sqrt_p, dk):
    n = noise.shape
    padded = np.zeros(tuple(2 * m for m in n))
    padded[:n[0], :n[1], :n[2]] = noise
    return np.ascontiguousarray(convolve_periodic(padded, h, sqrt_p, dk)[:n[0], :n[1], :n[2]])


def cubic_weights(t):
    """Lagrange weights through the nodes -1, 0, 1, 2, evaluated at t."""
    return np.array([-t * (t - 1) * (t - 2) / 6.0, (t + 1) * (t - 1) * (t - 2) / 2.0,
                     -(t + 1) * t * (t - 2) / 2.0, (t + 1) * t * (t - 1) / 6.0])


def tricubic_conservative(parent, off, n):
    """Parent-level field onto the nest of n fine cells at parent offset off."""
    out = np.asarray(parent, dtype=np.float64)
    for axis in range(3):
        idx = np.arange(n[axis])
        p = off[axis] + idx // 2
        odd = idx % 2 == 1
        first = np.where(odd, p - 1, p - 2)          # node -1 of the stencil
        t = np.where(odd, 0.25, 0.75)                # fine centre in node units
        w = cubic_weights(t)
        moved = np.moveaxis(out, axis, 0)
        acc = np.zeros((n[axis],) + moved.shape[1:])
        for s in range(4):
            acc += w[s].reshape((n[axis],) + (1,) * (moved.ndim - 1)) * moved[first + s]
        out = np.moveaxis(acc, 0, axis)
    region = tuple(slice(off[a], off[a] + n[a] // 2) for a in range(3))
    return out + inject(np.asarray(parent)[region] - children_mean(out))


def _region(nest):
    return tuple(slice(nest.off[a], nest.off[a] + nest.n[a] // 2) for a in range(3))


def level_noise(geom, seed):
    """The noise of every leaf level: stream l of the seed, nests constrained to
    their parent by Hoffman-Ribak."""
    mu = [white_noise(seed, int(np.prod(geom.base_n)), 0).reshape(tuple(geom.base_n))]
    for lvl, nest in enumerate(geom.nests, start=1):
        own = white_noise(seed, int(np.prod(nest.n)), lvl).reshape(tuple(nest.n))
        mu.append(own - inject(children_mean(own)) + inject(mu[-1][_region(nest)] / np.sqrt(8.0)))
    return mu


def multiscale(geom, seed, sqrt_p, dk):
    """delta on every leaf level of geom (base first), float64 C-ordered."""
    h = geom.box / geom.base_n[0]
    noise = level_noise(geom, seed)
    mu = noise[0]
    deltas = [convolve_periodic(mu, h, sqrt_p, dk)]
    region = _region
    ext = None
    if geom.nests:
        masked = mu.copy()
        masked[region(geom.nests[0])] = 0.0
        ext = convolve_periodic(masked, h, sqrt_p, dk)
    for lvl, nest in enumerate(geom.nests, start=1):
        h = h / 2.0
        own = noise[lvl]
        carried = tricubic_conservative(ext, nest.off, nest.n)
        deltas.append(convolve_isolated(own, h, sqrt_p, dk) + carried)
        if lvl < len(geom.nests):
            masked = own.copy()
            masked[region(geom.nests[lvl])] = 0.0
            ext = convolve_isolated(masked, h, sqrt_p, dk) + carried
        mu = own
    for lvl in range(len(geom.nests), 0, -1):
        deltas[lvl - 1][region(geom.nests[lvl - 1])] = children_mean(deltas[lvl])
    return deltas
