"""GB300-native Laplace-transform / flexible shifted-Krylov engine for
parabolic inverse problems (Bakhos, Saibaba & Kitanidis).

The compute path is the CUDA library liblt.so (C ABI in include/lt.h),
built in-tree by ``paper_1409_2556_gb300.build.build()``; this package only
marshals arguments.
"""
from .engine import Engine, LtError  # noqa: F401

__all__ = ["Engine", "LtError"]
