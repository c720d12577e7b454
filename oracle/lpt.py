"""Second-order LPT source and displacement gradient with finite differences.

* Displacement (eq. of Sec. 3.1.1): psi_a = -G_a^(n) phi, the Table-1
  gradient along axis a, on every leaf level with ghosts filled as in the
  solve.  The growth-factor normalisation is left to the caller.
* 2LPT source (Sec. 3.1.2): tau = sum_{i<j} (phi_,ii phi_,jj - phi_,ij^2),
  which equals the paper's -1/2 sum_{i,j}[(phi_,ij)^2 - phi_,ii phi_,jj]
  (the i = j terms cancel, each unordered pair appears twice).  phi_,ii is
  the 1D Table-1 second difference along i (so sum_i phi_,ii = L phi), and
  phi_,ij = G_i G_j phi, the composition of the two 1D gradients, which reads
  edge ghosts of nests.
* Second potential: L phi2 = tau on the composite grid, solved exactly like
  the first one (covered cells of tau = average of children, composite mean
  removed).  Positions follow x = q + D1 psi1 + (3/7) D1^2 psi2 with
  psi = -grad phi for both potentials (Scoccimarro 1998 sign convention; the
  paper's eq. for L and its D2 = 3/7 D+^2 differ in sign, see Sec. 3.1).
* Local Lagrangian density (Sec. 5.3): rho / rho_bar = 1 / det[delta_ij +
  dL_i/dq_j] from the same finite-difference Hessian, renormalised to unit
  composite mean.
"""

import numpy as np

from .hierarchy import Hierarchy, fill_ghosts, restrict
from .multigrid import composite_mean, solve, sync_covered
from .stencils import GRADIENT_1D, LAPLACIAN_1D


def load_potential(hier, phis):
    """Put the given per-leaf-level potentials into the hierarchy and sync covered cells."""
    for l, phi in zip(hier.leaf_levels(), phis):
        hier.levels[l].interior[...] = phi
    sync_covered(hier)


def gradient(hier, phis):
    """-G^(n) phi on every leaf level; returns a list of (psi_x, psi_y, psi_z)."""
    load_potential(hier, phis)
    out = []
    for l in hier.leaf_levels():
        lev = hier.levels[l]
        fill_ghosts(hier, l)
        w = GRADIENT_1D[lev.order]
        g = lev.g
        comps = []
        for axis in range(3):
            acc = np.zeros(lev.n)
            for s in range(-g, g + 1):
                if w[s + g] != 0.0:
                    acc += w[s + g] * lev.shifted(axis, s)
            comps.append(-acc / lev.h)
        out.append(tuple(comps))
    return out


def _shift2(lev, a, sa, b, sb):
    g, n = lev.g, lev.n
    sl = [slice(g, g + n[0]), slice(g, g + n[1]), slice(g, g + n[2])]
    sl[a] = slice(g + sa, g + sa + n[a])
    sl[b] = slice(g + sb, g + sb + n[b])
    return lev.u[tuple(sl)]


def second_derivatives(lev):
    """phi_,ii (i = 0..2) and phi_,ij (i < j) on the interior of a filled level."""
    wl = LAPLACIAN_1D[lev.order]
    wg = GRADIENT_1D[lev.order]
    g, h = lev.g, lev.h
    diag = []
    for a in range(3):
        acc = np.zeros(lev.n)
        for s in range(-g, g + 1):
            acc += wl[s + g] * lev.shifted(a, s)
        diag.append(acc / (h * h))
    mixed = {}
    for a in range(3):
        for b in range(a + 1, 3):
            acc = np.zeros(lev.n)
            for sa in range(-g, g + 1):
                if wg[sa + g] == 0.0:
                    continue
                for sb in range(-g, g + 1):
                    if wg[sb + g] == 0.0:
                        continue
                    acc += wg[sa + g] * wg[sb + g] * _shift2(lev, a, sa, b, sb)
            mixed[(a, b)] = acc / (h * h)
    return diag, mixed


def lpt2_source(hier, phis):
    """tau on every leaf level (before covered-cell averaging and mean removal)."""
    load_potential(hier, phis)
    out = []
    for l in hier.leaf_levels():
        fill_ghosts(hier, l, edges=True)
        diag, mixed = second_derivatives(hier.levels[l])
        tau = np.zeros(hier.levels[l].n)
        for a in range(3):
            for b in range(a + 1, 3):
                tau += diag[a] * diag[b] - mixed[(a, b)] ** 2
        out.append(tau)
    return out


def solve_2lpt(geom, phis1, **kw):
    """phi2 with L phi2 = tau(phi1) on the composite grid."""
    hier = Hierarchy(geom)
    tau = lpt2_source(hier, phis1)
    return solve(geom, tau, **kw)


def lpt_pipeline(geom, deltas, tol=1e-10, max_cycles=50, cycles=None):
    """phi1, phi2 and both displacement fields, as the library computes them."""
    phi1, info1 = solve(geom, deltas, tol=tol, max_cycles=max_cycles, cycles=cycles)
    phi2, info2 = solve_2lpt(geom, phi1, tol=tol, max_cycles=max_cycles, cycles=cycles)
    hier = Hierarchy(geom)
    psi1 = gradient(hier, phi1)
    psi2 = gradient(hier, phi2)
    return {"phi1": phi1, "phi2": phi2, "psi1": psi1, "psi2": psi2,
            "info1": info1, "info2": info2}


def lla_density(hier, phis1, phis2=None, a1=1.0, a2=0.0):
    """rho / rho_bar by the local Lagrangian approximation (Sec. 5.3, eq. for the
    gas density): 1 / det[delta_ij + dL_i/dq_j] with the displacement
    L = a1 psi1 + a2 psi2 = -grad(a1 phi1 + a2 phi2), so dL_i/dq_j = -Phi_,ij with
    Phi = a1 phi1 + a2 phi2 and Phi_,ij the finite differences of the 2LPT source.
    Covered cells hold the mean of their children; then the mass is restored by
    rho -> rho + (1 - <rho>), <.> the volume-weighted composite leaf mean (the
    paper's a-posteriori renormalisation, read as an additive shift)."""
    pot = [a1 * np.asarray(p1) + (a2 * np.asarray(p2) if phis2 is not None else 0.0)
           for p1, p2 in zip(phis1, phis2 if phis2 is not None else phis1)]
    load_potential(hier, pot)
    fields = []
    for l in hier.leaf_levels():
        fill_ghosts(hier, l, edges=True)
        diag, mixed = second_derivatives(hier.levels[l])
        jac = np.empty(tuple(hier.levels[l].n) + (3, 3))
        for a in range(3):
            jac[..., a, a] = 1.0 - diag[a]
            for b in range(a + 1, 3):
                jac[..., a, b] = -mixed[(a, b)]
                jac[..., b, a] = -mixed[(a, b)]
        fields.append(1.0 / np.linalg.det(jac))
    leaf = list(hier.leaf_levels())
    for i in range(len(leaf) - 1, 0, -1):
        fields[i - 1][hier.covered_region(leaf[i])] = restrict(fields[i])
    mean = composite_mean(hier, fields)
    return [f + (1.0 - mean) for f in fields]
