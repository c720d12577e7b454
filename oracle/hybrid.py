"""Hybrid Poisson solver correction (Sec. 3.5.2), test infrastructure only
(imported by tests/; nothing in the library path imports it).

The finite-difference solution of the finest level's own source f is replaced by
the exact k-space one: on the level's grid zero-padded to twice its size (f = 0
outside the level; a single periodic level is used as it is),
    correction_j = IFFT[ (i k_j / k^2 - G~_j / L~) FFT[f] ]   (paper, v = grad phi)
and, for the library's displacement psi = -G phi, the correction added to psi is
the negative of that: i (k_j / k^2) f~ + (G~_j / L~) f~ with numpy's exp(+ikx)
symbols G~_j = i g(k_j h) / h and L~ = sum_a L~(k_a h) / h^2 (Table 1).  The mode
k = 0 and, because the multiplier is odd in k_j, the Nyquist plane of axis j (even
sizes) get no correction; the result is the real part of the inverse transform,
restricted to the level's own cells.
"""

import numpy as np

from .stencils import gradient_symbol_1d, laplacian_symbol_1d


def hybrid_correction(f, h, order, pad=True):
    """The three components added to psi = -G phi on the level of source f."""
    f = np.asarray(f, dtype=np.float64)
    n = f.shape
    shape = tuple(2 * m for m in n) if pad else n
    grid = np.zeros(shape)
    grid[:n[0], :n[1], :n[2]] = f
    fk = np.fft.fftn(grid)
    theta = [2.0 * np.pi * np.fft.fftfreq(m) for m in shape]
    t = np.meshgrid(*theta, indexing="ij")
    k = [ta / h for ta in t]
    ksq = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
    lt = (laplacian_symbol_1d(order, t[0]) + laplacian_symbol_1d(order, t[1])
          + laplacian_symbol_1d(order, t[2])) / (h * h)
    zero = ksq == 0.0
    ksq[zero] = 1.0
    lt[zero] = 1.0
    out = []
    for j in range(3):
        gt = 1j * gradient_symbol_1d(order, t[j]) / h      # G~_j = i g / h
        mult = 1j * k[j] / ksq + gt / lt
        mult[zero] = 0.0
        if shape[j] % 2 == 0:
            sl = [slice(None)] * 3
            sl[j] = shape[j] // 2
            mult[tuple(sl)] = 0.0
        corr = np.fft.ifftn(mult * fk).real
        out.append(np.ascontiguousarray(corr[:n[0], :n[1], :n[2]]))
    return out
