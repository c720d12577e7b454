"""Levels, ghost zones and inter-level transfer for the composite (nested) grid.

Level structure (Sec. 3.2-3.3, Fig. 3): levels 0..B-1 are the full periodic
multigrid coarsenings of the base grid B (refinement factor 2; halving stops
once some side is odd, no side exceeds 8, or a halved side would be narrower
than the ghost width); levels B+1.. are nested rectangular patches, each
inside its parent, at twice the parent's resolution.  Every level stores u
with a ghost shell of width g = n/2 (n = order of the FD Laplacian).  Arrays
are float64, [x][y][z], z fastest.

Transfers (Sec. 3.2 step 4-5, 8 and the closing paragraph): restriction is
the average of the 8 children, prolongation is straight injection into the 8
children; on nests both act only on the covered region (Sec. 3.3).

Ghosts: periodic wrap on full levels (Sec. 3.2, "enforce periodic boundary
conditions whenever u is changed").  On a nest (Sec. 3.3): a degree-n
polynomial through parent values parallel to the face, then a degree-n
polynomial normal to the face through those intermediate values and fine
interior values, then flux matching: the face flux of order n-1 (Table 2) is
evaluated on the parent and on the 4 fine faces beneath each parent face
element, and the difference is added to the ghost values that enter the
fine flux, so that the mean of the 4 fine fluxes equals the parent flux.
"""

import numpy as np

from .stencils import (FLUX_1D, LAPLACIAN_1D, ghost_width, normal_weights,
                       tangential_weights)


class Level:
    def __init__(self, n, h, order, periodic, off=None, has_source=True):
        self.n = tuple(int(v) for v in n)
        self.h = float(h)
        self.order = order
        self.g = ghost_width(order)
        self.periodic = periodic
        self.off = None if off is None else tuple(int(v) for v in off)
        g = self.g
        self.u = np.zeros(tuple(v + 2 * g for v in self.n))
        self.f = np.zeros(self.n) if has_source else None
        self.ffas = np.zeros(self.n)
        self.ubar = None
        i, j, k = np.meshgrid(*[np.arange(v) for v in self.n], indexing="ij")
        self.colour = (i + j + k) % 2

    @property
    def interior(self):
        g, n = self.g, self.n
        return self.u[g:g + n[0], g:g + n[1], g:g + n[2]]

    def shifted(self, axis, s, arr=None):
        """View of the interior shifted by s cells along axis (s may reach the ghosts)."""
        a = self.u if arr is None else arr
        g, n = self.g, self.n
        sl = [slice(g, g + n[0]), slice(g, g + n[1]), slice(g, g + n[2])]
        sl[axis] = slice(g + s, g + s + n[axis])
        return a[tuple(sl)]


class Hierarchy:
    """Full coarsening chain below the base, the base, and the chain of nests."""

    def __init__(self, geom):
        self.order = geom.order
        self.box = float(geom.box)
        base_n = tuple(geom.base_n)
        chain = [base_n]
        g = ghost_width(self.order)
        # coarsen while every side is even, some side exceeds 8, and every side of the
        # coarser level still holds a full ghost width
        while (all(v % 2 == 0 for v in chain[-1]) and max(chain[-1]) > 8
               and min(chain[-1]) // 2 >= g):
            chain.append(tuple(v // 2 for v in chain[-1]))
        chain.reverse()
        self.base = len(chain) - 1
        self.levels = []
        for idx, n in enumerate(chain):
            h = self.box / n[0]
            self.levels.append(Level(n, h, self.order, True, off=None,
                                     has_source=(idx == self.base)))
        h = self.box / base_n[0]
        for nest in geom.nests:
            h = h / 2.0
            self.levels.append(Level(nest.n, h, self.order, False, off=nest.off))

    @property
    def finest(self):
        return len(self.levels) - 1

    def covered_region(self, l):
        """Slice of level l-1's interior covered by level l."""
        lev = self.levels[l]
        off = lev.off if lev.off is not None else (0, 0, 0)
        return tuple(slice(off[a], off[a] + lev.n[a] // 2) for a in range(3))

    def uncovered_mask(self, l):
        mask = np.ones(self.levels[l].n, dtype=bool)
        if l < self.finest:
            mask[self.covered_region(l + 1)] = False
        return mask

    def leaf_levels(self):
        return range(self.base, len(self.levels))


def restrict(fine):
    """Average over the 8 children of each parent cell."""
    n = fine.shape
    return fine.reshape(n[0] // 2, 2, n[1] // 2, 2, n[2] // 2, 2).mean(axis=(1, 3, 5))


def inject(coarse):
    """Straight injection of each parent value into its 8 children."""
    return np.repeat(np.repeat(np.repeat(coarse, 2, axis=0), 2, axis=1), 2, axis=2)


def laplacian(lev, arr=None):
    """L^(n) u on the interior: sum over axes of the 1D Table-1 stencil."""
    w = LAPLACIAN_1D[lev.order]
    g = lev.g
    out = np.zeros(lev.n)
    for axis in range(3):
        for s in range(-g, g + 1):
            out += w[s + g] * lev.shifted(axis, s, arr)
    return out / (lev.h * lev.h)


def fill_periodic(lev):
    u, g, n = lev.u, lev.g, lev.n
    for axis in range(3):
        lo = [slice(None)] * 3
        src = [slice(None)] * 3
        lo[axis] = slice(0, g)
        src[axis] = slice(n[axis], n[axis] + g)
        u[tuple(lo)] = u[tuple(src)]
        hi = [slice(None)] * 3
        src2 = [slice(None)] * 3
        hi[axis] = slice(n[axis] + g, n[axis] + 2 * g)
        src2[axis] = slice(g, 2 * g)
        u[tuple(hi)] = u[tuple(src2)]


def _interp_axis(values, axis, fine_idx, off, weights, half):
    """Along `axis` of `values` (parent index space), evaluate the degree-n
    Lagrange interpolant centred on the parent cell off + floor(i/2) at the
    centre of fine cell i, for every i in fine_idx."""
    fine_idx = np.asarray(fine_idx)
    p = off + np.floor_divide(fine_idx, 2)
    par = np.mod(fine_idx, 2)
    moved = np.moveaxis(values, axis, 0)
    out = np.zeros((len(fine_idx),) + moved.shape[1:])
    for s in range(-half, half + 1):
        w = np.where(par == 1, weights[1][s + half], weights[0][s + half])
        out += w.reshape((-1,) + (1,) * (moved.ndim - 1)) * moved[p + s]
    return np.moveaxis(out, 0, axis)


def fill_coarse_fine(hier, l, edges=False, flux_fix=True):
    """Ghost zones of nest l from its parent (Sec. 3.3).

    Face ghosts: tangential interpolation on parent data, normal interpolation
    with fine interior data, then flux matching.  With edges=True the edge and
    corner ghosts (needed only by the mixed derivatives of the 2LPT source)
    are filled by tensor degree-n interpolation of parent data alone.

    Two-way interface (Sec. 3.3): the covered parent cells are first set to the
    average of their current children, so that the parent flux on every
    coarse-fine face is the flux of the composite solution.  (Taking the
    parent flux from covered values that lag the fine solution slows the
    composite V-cycle from ~15x to ~4.5x residual reduction per cycle.)"""
    lev = hier.levels[l]
    par = hier.levels[l - 1]
    par.interior[hier.covered_region(l)] = restrict(lev.interior)
    U = par.interior
    order, g, n, off = lev.order, lev.g, lev.n, lev.off
    half = order // 2
    tw = tangential_weights(order)
    cw, fw = normal_weights(order)
    F = FLUX_1D[order]
    h, H = lev.h, par.h
    u = lev.u
    for a in range(3):
        b, c = [x for x in range(3) if x != a]
        for side in (0, 1):
            # intermediate values at the parent centres outside the face
            inter = []
            for m in range(half):
                pn = off[a] - 1 - m if side == 0 else off[a] + n[a] // 2 + m
                slab = np.take(U, pn, axis=a)  # 2D array over (b, c) in parent index space
                t = _interp_axis(slab, 0, np.arange(n[b]), off[b], tw, half)
                t = _interp_axis(t, 1, np.arange(n[c]), off[c], tw, half)
                inter.append(t)
            # fine interior values next to the face: q = 0 .. half
            fine = []
            for q in range(half + 1):
                idx = g + q if side == 0 else g + n[a] - 1 - q
                fine.append(_face_plane(u, a, idx, g, n))
            ghosts = []
            for m in range(g):
                val = np.zeros((n[b], n[c]))
                for q in range(half):
                    val += cw[m, q] * inter[q]
                for q in range(half + 1):
                    val += fw[m, q] * fine[q]
                ghosts.append(val)
            for m in range(g):
                idx = g - 1 - m if side == 0 else g + n[a] + m
                _set_face_plane(u, a, idx, g, n, ghosts[m])
            if not flux_fix:
                continue
            # fine flux through the face, per fine column (cells face-half .. face+half-1)
            face = g if side == 0 else g + n[a]
            ff = np.zeros((n[b], n[c]))
            for s in range(order):
                ff += F[s] * _face_plane(u, a, face - half + s, g, n)
            ff /= h
            # parent flux through the same face, per parent face element
            pface = off[a] if side == 0 else off[a] + n[a] // 2
            tb = slice(off[b], off[b] + n[b] // 2)
            tc = slice(off[c], off[c] + n[c] // 2)
            fc = np.zeros((n[b] // 2, n[c] // 2))
            for s in range(order):
                plane = np.take(U, pface - half + s, axis=a)
                fc += F[s] * plane[tb, tc]
            fc /= H
            mean_fine = ff.reshape(n[b] // 2, 2, n[c] // 2, 2).mean(axis=(1, 3))
            dF = fc - mean_fine
            ghost_coef = F[:half].sum() if side == 0 else F[half:].sum()
            shift = np.repeat(np.repeat(dF * h / ghost_coef, 2, axis=0), 2, axis=1)
            for m in range(g):
                idx = g - 1 - m if side == 0 else g + n[a] + m
                _set_face_plane(u, a, idx, g, n, _face_plane(u, a, idx, g, n) + shift)
    if edges:
        _fill_edges(lev, U, tw, half)


def _face_plane(u, axis, idx, g, n):
    """Plane of u at padded index idx along axis, restricted to the interior
    range of the two tangential axes."""
    sl = [slice(g, g + n[0]), slice(g, g + n[1]), slice(g, g + n[2])]
    sl[axis] = idx
    return u[tuple(sl)].copy()


def _set_face_plane(u, axis, idx, g, n, val):
    sl = [slice(g, g + n[0]), slice(g, g + n[1]), slice(g, g + n[2])]
    sl[axis] = idx
    u[tuple(sl)] = val


def _fill_edges(lev, U, tw, half):
    """Edge and corner ghosts: tensor interpolation of parent data only."""
    g, n, off = lev.g, lev.n, lev.off
    t = U
    for a in range(3):
        t = _interp_axis(t, a, np.arange(-g, n[a] + g), off[a], tw, half)
    outside = np.zeros(t.shape, dtype=np.int8)
    for a in range(3):
        idx = np.arange(-g, n[a] + g)
        ax = ((idx < 0) | (idx >= n[a])).astype(np.int8)
        shape = [1, 1, 1]
        shape[a] = -1
        outside = outside + ax.reshape(shape)
    sel = outside >= 2
    lev.u[sel] = t[sel]


def fill_ghosts(hier, l, edges=False, flux_fix=True):
    lev = hier.levels[l]
    if lev.periodic:
        fill_periodic(lev)
    else:
        fill_coarse_fine(hier, l, edges=edges, flux_fix=flux_fix)
