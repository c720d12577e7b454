"""GB300-native nested-grid Poisson / 2LPT / displacement solver (MUSIC hot path).

The compute path is the CUDA library libmgic.so (C ABI in include/mg.h); this
package holds its sources (csrc/), its build script and a thin ctypes binding.
"""

from .mg import (MG_FP64, MG_MIXED, Batch, Field, Hierarchy, MGConfig, MGError, MGInfo,
                 config_from_geometry, load_library, make_config, validate, white_noise,
                 workspace_bytes)

__all__ = ["MG_FP64", "MG_MIXED", "Batch", "Field", "Hierarchy", "MGConfig", "MGError", "MGInfo",
           "config_from_geometry", "load_library", "make_config", "validate", "white_noise",
           "workspace_bytes"]
