"""GB300-native label-propagation refinement for hypergraph partitioning.

The compute runs in libhgp.so (hand-written CUDA for sm_103a behind the C ABI declared in
include/hgp.h).  This package only marshals arguments to it; there is no CPU fallback: if
the library is not built, every entry point raises.
"""
from .native import (HGP, Batch, Coarse, HGPError, STAT_FIELDS, default_options, library_path,  # noqa: F401
                     load_library, strerror)

__all__ = ["HGP", "Batch", "Coarse", "HGPError", "STAT_FIELDS", "default_options", "library_path",
           "load_library", "strerror"]
