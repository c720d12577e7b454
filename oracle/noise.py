"""Oracle for the GPU density generator (test infrastructure only: imported by
tests/, __graft_entry__.smoke() and bench.py's CPU baseline; nothing in the
library path imports it).

The paper draws the density field from Gaussian white noise convolved with the
transfer function, Sec. 2.1: delta(k) = sqrt(P(k)) mu(k).  The generator that
the GPU implements needs random numbers that both sides can draw, so it uses one
counter-based generator from its published definition:

* Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011, "Parallel random numbers: as
  easy as 1, 2, 3", SC11): a 4 x 32-bit counter and a 2 x 32-bit key; each of the
  10 rounds multiplies counter words 0 and 2 by the constants 0xD2511F53 and
  0xCD9E8D57, and mixes the high halves with words 1, 3 and the key; the key is
  bumped by the Weyl constants 0x9E3779B9 and 0xBB67AE85 before every round but
  the first.
* Normal deviates by the Box-Muller transform of two uniforms in (0, 1), each
  built from two 32-bit outputs (27 + 26 bits, offset by half a unit in the
  last place so that 0 and 1 never occur).

Element i of the noise comes from pair index q = i // 2: counter (q mod 2^32,
q div 2^32, stream, 0), key (seed mod 2^32, seed div 2^32); outputs x0..x3 give
u1 = ((x0 >> 5) 2^26 + (x1 >> 6) + 1/2) / 2^53 and u2 likewise from x2, x3;
element 2q = r cos(2 pi u2), element 2q + 1 = r sin(2 pi u2), r = sqrt(-2 ln u1).

The periodic field is delta = IFFT[A(|k|) FFT[noise]] (numpy's unnormalised
forward and 1/N inverse transforms), with A linearly interpolated from a table
sampled at |k| = t dk, zero beyond it and at k = 0 (Sec. 2.1: the amplitude is
sqrt(P(k)/h^3) in these units).
"""

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_LO = np.uint64(0xFFFFFFFF)


def philox4x32_10(counter, key):
    """counter: uint32 array (4, n); key: uint32 array (2, n) (or (2,) broadcast).
    Returns the uint32 array (4, n) of outputs."""
    x = [np.asarray(c, dtype=np.uint32).copy() for c in counter]
    k0 = np.asarray(key[0], dtype=np.uint32).copy()
    k1 = np.asarray(key[1], dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        for r in range(10):
            if r:
                k0 = k0 + _W0
                k1 = k1 + _W1
            p0 = _M0 * x[0].astype(np.uint64)
            p1 = _M1 * x[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _LO).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _LO).astype(np.uint32)
            x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return np.stack(x)


def uniform53(a, b):
    """Uniform in (0, 1) from two 32-bit words: 27 bits of a, 26 bits of b."""
    hi = (np.asarray(a, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    lo = (np.asarray(b, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (hi * 67108864.0 + lo + 0.5) / 9007199254740992.0


def white_noise(seed, n, stream=0):
    """n standard normal deviates, element i from pair index i // 2 (see header);
    stream goes into counter word 2 (0 for a single field; the level of a nest)."""
    seed = int(seed)
    pairs = (int(n) + 1) // 2
    q = np.arange(pairs, dtype=np.uint64)
    ctr = np.stack([(q & _LO).astype(np.uint32), (q >> np.uint64(32)).astype(np.uint32),
                    np.full(pairs, int(stream) & 0xFFFFFFFF, np.uint32), np.zeros(pairs, np.uint32)])
    key = (np.uint32(seed & 0xFFFFFFFF), np.uint32((seed >> 32) & 0xFFFFFFFF))
    x = philox4x32_10(ctr, key)
    u1 = uniform53(x[0], x[1])
    u2 = uniform53(x[2], x[3])
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * pairs)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:n]


def kmag(shape, h):
    """|k| on the FFT grid of a periodic box of cubic cells of side h."""
    axes = [2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in shape]
    kx, ky, kz = np.meshgrid(*axes, indexing="ij")
    return np.sqrt(kx * kx + ky * ky + kz * kz)


def amplitude(k, amp, dk):
    """Linear interpolation of the table amp[t] at |k| = t dk; 0 beyond the table."""
    amp = np.asarray(amp, dtype=np.float64)
    t = np.asarray(k) / dk
    out = np.interp(t, np.arange(amp.size, dtype=np.float64), amp)
    out[t > amp.size - 1] = 0.0
    return out


def gaussian_field(noise, h, amp, dk):
    """delta = IFFT[A(|k|) FFT[noise]], A(0) = 0, on the periodic grid of noise."""
    a = amplitude(kmag(noise.shape, h), amp, dk)
    a.flat[0] = 0.0
    return np.ascontiguousarray(np.fft.ifftn(np.fft.fftn(noise) * a).real)
