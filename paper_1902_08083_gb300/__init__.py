"""GB300-native (sm_103a) implementation of the TREVR hot path.

TREVR (Grond, Woods, Wadsley & Couchman 2019, arXiv:1902.08083) is a
tree-based reverse ray tracer for radiative transfer. The CUDA library
``libtrevr.so`` (C ABI in ``include/trevr.h``) builds the radiation tree and
computes the flux at every sink; ``trevr.py`` is a thin ctypes binding.
"""
from .trevr import (Batch, Tree, TrevrError, TrevrFlux, build_tree, check, compute_flux,  # noqa: F401
                    compute_flux_backward, load_library, make_params, trevr_flux)

__all__ = ["Batch", "Tree", "TrevrError", "TrevrFlux", "build_tree", "check", "compute_flux",
           "compute_flux_backward", "load_library", "make_params", "trevr_flux"]
