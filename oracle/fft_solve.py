"""Exact solution of the discrete periodic problem by the DFT.

On a single periodic grid the multigrid iteration converges to the unique
zero-mean solution of L^(n) phi = f.  L^(n) is diagonal in Fourier space with
eigenvalue sum_a L~(k_a h) / h^2 (Table 1, bottom rows), so
phi^(k) = f^(k) / L~(k), phi^(0) = 0; the gradient multiplies each mode by
+i g(k_a h) / h (Table 1 gradient symbol in numpy's exp(+ikx) convention).
The same solve is the coarsest-level step of the V-cycle (reading of Sec. 3.2
step 1: the coarsening stops at a side of at most 8 or an odd side, where the
level is solved exactly instead of setting u = 0 on a single cell).
"""

import numpy as np

from .stencils import gradient_symbol_1d, laplacian_symbol_1d


def _theta(n):
    return 2.0 * np.pi * np.fft.fftfreq(n)


def laplacian_symbol(shape, h, order):
    tx, ty, tz = np.meshgrid(*[_theta(n) for n in shape], indexing="ij")
    return (laplacian_symbol_1d(order, tx) + laplacian_symbol_1d(order, ty)
            + laplacian_symbol_1d(order, tz)) / (h * h)


def exact_solve(f, h, order):
    lam = laplacian_symbol(f.shape, h, order)
    fk = np.fft.fftn(f)
    lam[0, 0, 0] = 1.0
    phik = fk / lam
    phik[0, 0, 0] = 0.0
    return np.fft.ifftn(phik).real


def spectral_gradient(phi, h, order):
    """The three components of -G^(n) phi on a periodic grid."""
    phik = np.fft.fftn(phi)
    out = []
    for axis in range(3):
        shape = [1, 1, 1]
        shape[axis] = -1
        g = gradient_symbol_1d(order, _theta(phi.shape[axis])).reshape(shape) / h
        out.append(-np.fft.ifftn(1j * g * phik).real)
    return out
