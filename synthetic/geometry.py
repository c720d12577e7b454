"""Hierarchy geometries of the stand-in workloads.

A hierarchy is a periodic base grid plus a chain of nested rectangular
patches, each at twice the resolution of its parent (Sec. 3.3; Fig. 3).  A
nest is given by its size in its own cells (even on every axis) and by its
origin in PARENT cells; it covers parent cells [off, off + n/2).
"""

from dataclasses import dataclass, field
from typing import List, Tuple

import numpy as np

Int3 = Tuple[int, int, int]


@dataclass(frozen=True)
class NestSpec:
    n: Int3
    off: Int3


@dataclass(frozen=True)
class Geometry:
    base_n: Int3
    box: float
    order: int
    nests: Tuple[NestSpec, ...] = field(default_factory=tuple)

    @property
    def n_levels(self) -> int:
        return 1 + len(self.nests)

    def level_cells(self) -> int:
        """Sum over base and nests of the interior cell count."""
        total = int(np.prod(self.base_n))
        for nest in self.nests:
            total += int(np.prod(nest.n))
        return total


def level_shapes(geom: Geometry) -> List[Int3]:
    return [tuple(geom.base_n)] + [tuple(n.n) for n in geom.nests]


def config_unigrid64() -> Geometry:
    """Single periodic 64^3 level, 7-point (order 2) Laplacian; box of unit length."""
    return Geometry((64, 64, 64), 1.0, 2, ())


def config_zoom2(base: int = 128, nest: int = 128, order: int = 6, box: float = 100.0) -> Geometry:
    """Base grid plus one centred nest at twice the resolution."""
    off = (base - nest // 2) // 2
    return Geometry((base,) * 3, box, order, (NestSpec((nest,) * 3, (off,) * 3),))


def config_deep_zoom(seed: int = 3, base: int = 128, nest: int = 128, levels: int = 4,
                     jitter: int = 16, order: int = 6, box: float = 100.0) -> Geometry:
    """Base plus `levels` nests, each centred in its parent with a seeded offset jitter."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nests = []
    parent = base
    for _ in range(levels):
        centred = (parent - nest // 2) // 2
        off = tuple(int(centred + rng.integers(-jitter, jitter + 1)) for _ in range(3))
        nests.append(NestSpec((nest,) * 3, off))
        parent = nest
    return Geometry((base,) * 3, box, order, tuple(nests))


def small_zoom(base: int = 32, nests=((32, 8),), order: int = 2, box: float = 1.0) -> Geometry:
    """Cubic base plus a chain of cubic nests given as (side, offset) in parent cells."""
    return Geometry((base,) * 3, box, order,
                    tuple(NestSpec((n,) * 3, (o,) * 3) for n, o in nests))


def random_hierarchy(rng, bases=(32, 48, 64, 96, 128), max_nests: int = 3, order: int = 6,
                     box: float = 100.0) -> Geometry:
    """One hierarchy of the batched workload: base side drawn uniformly from `bases`,
    0..max_nests nests of side 0.5-1.0 x base (even, clamped to fit the parent with a
    margin of `order` parent cells), uniform random offsets."""
    base = int(rng.choice(bases))
    count = int(rng.integers(0, max_nests + 1))
    margin = order
    nests = []
    parent = base
    for _ in range(count):
        side = int(round(rng.uniform(0.5, 1.0) * base))
        side -= side % 2
        side = min(side, 2 * (parent - 2 * margin))
        side -= side % 2
        if side < 8:
            break
        hi = parent - side // 2 - margin
        off = tuple(int(rng.integers(margin, hi + 1)) for _ in range(3))
        nests.append(NestSpec((side,) * 3, off))
        parent = side
    return Geometry((base,) * 3, box, order, tuple(nests))


def config_batch(seed: int = 4, count: int = 64, order: int = 6) -> List[Geometry]:
    rng = np.random.Generator(np.random.PCG64(seed))
    return [random_hierarchy(rng, order=order) for _ in range(count)]
