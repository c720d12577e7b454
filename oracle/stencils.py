"""Finite-difference operators of Table 1 and Table 2, their Fourier symbols,
and Lagrange interpolation weights.

Table 1 (Sec. 3.2): 1D Laplacian L and gradient G of order n = 2, 4, 6 and
their Fourier transforms.  The 3D Laplacian is the sum of the 1D second
differences along x, y and z (7/13/19 points); the 3D gradient component a is
the 1D gradient along axis a.

Table 2 (Sec. 3.3): face-flux operators F of order n-1.  The printed rows do
not share one sign convention (convolving [-1 1] with the printed order-3 and
order-5 rows gives the NEGATED Laplacian, the order-1 row gives +[1 -2 1]).
The oracle defines F on face i+1/2 by F_{i+1/2} - F_{i-1/2} = L_i, which fixes
the sign of every row; tests check this telescoping against Table 1.
"""

from fractions import Fraction

import numpy as np

ORDERS = (2, 4, 6)

# Table 1, top rows: stencil weights on offsets -n/2 .. n/2 (in units of 1/h^2 and 1/h).
LAPLACIAN_1D = {
    2: np.array([1.0, -2.0, 1.0]),
    4: np.array([-1.0, 16.0, -30.0, 16.0, -1.0]) / 12.0,
    6: np.array([2.0, -27.0, 270.0, -490.0, 270.0, -27.0, 2.0]) / 180.0,
}
GRADIENT_1D = {
    2: np.array([-1.0, 0.0, 1.0]) / 2.0,
    4: np.array([1.0, -8.0, 0.0, 8.0, -1.0]) / 12.0,
    6: np.array([-1.0, 9.0, -45.0, 0.0, 45.0, -9.0, 1.0]) / 60.0,
}

# Table 2 with the sign fixed by telescoping: weights on cells i-n/2+1 .. i+n/2
# for the face i+1/2 (in units of 1/h).
FLUX_1D = {
    2: np.array([-1.0, 1.0]),
    4: np.array([1.0, -15.0, 15.0, -1.0]) / 12.0,
    6: np.array([-2.0, 25.0, -245.0, 245.0, -25.0, 2.0]) / 180.0,
}


def ghost_width(order: int) -> int:
    return order // 2


def laplacian_symbol_1d(order: int, theta):
    """Table 1, bottom rows: L~(theta) for h = 1 (theta = k h)."""
    c = np.cos
    t = np.asarray(theta, dtype=np.float64)
    if order == 2:
        return -2.0 * (1.0 - c(t))
    if order == 4:
        return -(c(2 * t) - 16.0 * c(t) + 15.0) / 6.0
    if order == 6:
        return -(-2.0 * c(3 * t) + 27.0 * c(2 * t) - 270.0 * c(t) + 245.0) / 90.0
    raise ValueError(order)


def gradient_symbol_1d(order: int, theta):
    """Magnitude g(theta) of the gradient symbol for h = 1.

    Table 1 prints -i g(k) in the convention exp(-ikx) for the inverse
    transform; with numpy's inverse transform exp(+ikx) a derivative acts as
    +i k, so the gradient multiplies a mode by +i g(theta)."""
    s = np.sin
    t = np.asarray(theta, dtype=np.float64)
    if order == 2:
        return s(t)
    if order == 4:
        return (8.0 * s(t) - s(2 * t)) / 6.0
    if order == 6:
        return (45.0 * s(t) - 9.0 * s(2 * t) + s(3 * t)) / 30.0
    raise ValueError(order)


def lagrange_weights(nodes, x):
    """Exact weights w_j with p(x) = sum_j w_j p(nodes_j) for every polynomial of
    degree < len(nodes); nodes and x are rationals (Fractions or ints)."""
    nodes = [Fraction(v) for v in nodes]
    x = Fraction(x)
    out = []
    for j, xj in enumerate(nodes):
        w = Fraction(1)
        for m, xm in enumerate(nodes):
            if m != j:
                w *= (x - xm) / (xj - xm)
        out.append(w)
    return out


def tangential_weights(order: int):
    """Coarse-only interpolation parallel to a coarse-fine face (Sec. 3.3).

    Degree-n polynomial through the n+1 parent cells centred on the parent
    cell that contains the fine cell, evaluated at the fine centre, which lies
    1/4 parent cell below (even fine index) or above (odd fine index) the
    parent centre.  Returns {0: weights for even, 1: weights for odd} on parent
    offsets -n/2..n/2."""
    half = order // 2
    nodes = list(range(-half, half + 1))
    return {0: np.array([float(w) for w in lagrange_weights(nodes, Fraction(-1, 4))]),
            1: np.array([float(w) for w in lagrange_weights(nodes, Fraction(1, 4))])}


def normal_weights(order: int):
    """Interpolation normal to a coarse-fine face (Sec. 3.3).

    Positions in fine cells measured from the face, positive into the nest:
    n/2 coarse intermediate values at -1, -3, -5, ... (parent centres outside
    the face), n/2+1 fine interior centres at 1/2, 3/2, ...; the degree-n
    polynomial is evaluated at the g = n/2 ghost centres -1/2, -3/2, ...
    Returns (coarse_w, fine_w) with shape (g, n/2) and (g, n/2+1); row m is
    ghost layer m (m = 0 is adjacent to the face)."""
    half = order // 2
    coarse_nodes = [Fraction(-(2 * m + 1)) for m in range(half)]
    fine_nodes = [Fraction(2 * q + 1, 2) for q in range(half + 1)]
    nodes = coarse_nodes + fine_nodes
    cw = np.zeros((half, half))
    fw = np.zeros((half, half + 1))
    for m in range(half):
        w = lagrange_weights(nodes, Fraction(-(2 * m + 1), 2))
        cw[m] = [float(v) for v in w[:half]]
        fw[m] = [float(v) for v in w[half:]]
    return cw, fw
