"""Seeded synthetic inputs for the nested-grid Poisson / 2LPT path.

This package is shared by the CPU oracle's tests, the GPU parity tests and
the benchmark.  It holds no arithmetic of the solver itself: only white
noise, power spectra, the multi-scale density convolution that produces the
source field delta on every level (Sec. 2.1-2.3 of Hahn & Abel 2011), and the
hierarchy geometries of the stand-in workloads.
"""

from .geometry import Geometry, NestSpec, config_unigrid64, config_zoom2, config_deep_zoom, \
    config_batch, small_zoom, level_shapes
from .density import white_noise, make_delta, make_delta_powerlaw
from .spectra import Cosmology, BBKSPower, PowerLaw

__all__ = [
    "Geometry", "NestSpec", "config_unigrid64", "config_zoom2", "config_deep_zoom",
    "config_batch", "small_zoom", "level_shapes", "white_noise", "make_delta",
    "make_delta_powerlaw", "Cosmology", "BBKSPower", "PowerLaw",
]
