"""Gauss-Legendre spherical harmonic transforms for NVIDIA GB300 (sm_103a).

The transforms of Schaeffer's SHTns paper (arXiv:1202.6522) as hand-written
CUDA kernels behind a C ABI (include/sht.h, libsht.so).  ``SHT`` is the torch
front end; ``_capi`` is the ctypes binding with the C names; ``build.build()``
compiles the library in-tree.
"""
from __future__ import annotations

__all__ = ["SHT", "UnevenBatch", "build", "synthetic"]


def __getattr__(name):
    if name == "SHT":
        from .transform import SHT
        return SHT
    if name == "UnevenBatch":
        from .transform import UnevenBatch
        return UnevenBatch
    raise AttributeError(name)
