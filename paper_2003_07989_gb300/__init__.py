"""GB300-native Vietoris-Rips persistence barcodes over Z/2.

The computation runs in librpp.so (CUDA kernels for sm_103a plus native host
code), declared in include/rpp.h. This package is the thin Python binding:

  rpp_barcodes(points_or_D, max_dim, threshold, ...)   one instance
  rpp_barcodes_batched([clouds], max_dim, ...)          many instances per call
  Server(...).submit / .poll                            continuous batching
  rips_persistence / total_persistence                  autograd (rpp_barcodes_backward)

The build step is ``paper_2003_07989_gb300.build.build()``. Importing the
binding functions raises if the library was not built.
"""
from ._native import RppError
from .api import (Barcodes, Context, Server, default_context, rpp_apparent_census,
                  rpp_barcodes, rpp_barcodes_batched, rpp_distance_matrix, rpp_filtration,
                  rpp_l2_read_probe)

__all__ = ["Barcodes", "Context", "RppError", "Server", "default_context", "rpp_apparent_census",
           "rpp_barcodes", "rpp_barcodes_batched", "rpp_distance_matrix", "rpp_filtration",
           "rpp_l2_read_probe", "rips_persistence",
           "total_persistence"]


def __getattr__(name):
    if name in ("rips_persistence", "total_persistence", "RipsPersistence"):
        from . import autograd
        return getattr(autograd, name)
    raise AttributeError(name)
