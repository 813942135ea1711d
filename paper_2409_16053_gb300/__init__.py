"""GB300-native hydro stage of AthenaK (arXiv 2409.16053): one Runge-Kutta stage of the
Godunov finite-volume update for 3D adiabatic Newtonian hydrodynamics on a mesh of
MeshBlocks, as hand-written CUDA for sm_103a behind a C-ABI (include/ak.h).

    from paper_2409_16053_gb300 import build; build.build()   # nvcc -> _build/libak.so
    from paper_2409_16053_gb300 import ak                     # ctypes binding
"""
from . import build  # noqa: F401

__all__ = ["build"]
