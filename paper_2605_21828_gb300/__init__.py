"""GB300-native butterfly-accelerated manifold harmonic transform (BF-MHT).

The library (``libmht.so``: FP64 host build + sm_103a CUDA apply kernels behind the C ABI
in ``include/mht.h``) is built in-tree by :func:`paper_2605_21828_gb300.build.build_library`.
"""
from .api import Batch, Plan, analyze, phi_entries, synthesize  # noqa: F401
from ._lib import MhtError, load  # noqa: F401

__all__ = ["Plan", "Batch", "synthesize", "analyze", "phi_entries", "MhtError", "load"]
