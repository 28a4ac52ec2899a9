"""GB300 (sm_103a) photoacoustic forward/adjoint operators for DIP and TV reconstruction.

The operators themselves live in the CUDA library ``libpatgpu.so`` (C ABI in
``include/pat.h``); this package is its thin Python binding plus the
reconstruction loops that call it.  Importing the package does not load the
library; the first operator call does, and fails loudly if it is missing.
"""
from .api import Geometry, PatPlan, arc, full_circle  # noqa: F401

__all__ = ["Geometry", "PatPlan", "arc", "full_circle"]
