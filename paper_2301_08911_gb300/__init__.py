"""GB300 (sm_103a) solver for the per-iteration hot path of density-based inverse
homogenization (arXiv 2301.08911): 6 periodic cell problems by multigrid-preconditioned
CG, the homogenised tensor C^H, sensitivities, periodic density filter and OC update.

The compute path is libhomo.so (CUDA, C ABI in include/homo.h); this package only builds
it and binds it. Importing the package does not load the library; `binding` does, and
fails loudly when it has not been built.
"""
from . import build  # noqa: F401

__all__ = ["build", "binding"]
