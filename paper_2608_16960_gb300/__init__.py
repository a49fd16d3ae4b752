"""GB300-native spherical-grid tomographic projector (TomoSphero, arxiv 2608.16960).

The compute path is libtsp.so (hand-written CUDA for sm_103a behind the C ABI
in include/tsp.h). This package holds the build step, the ctypes binding and
the seeded synthetic-input generators; torch supplies device memory, streams
and autograd plumbing only.
"""
from __future__ import annotations

__all__ = ["Grid", "Geometry", "Operator", "ProjectorFn", "tsp_forward", "tsp_adjoint", "build"]


def build(force: bool = False) -> str:
    from .nvbuild import build as _b
    return _b(force=force)


def __getattr__(name):
    if name in ("Grid", "Geometry", "Operator", "ProjectorFn", "tsp_forward", "tsp_adjoint", "tsp_device_status"):
        from . import projector
        return getattr(projector, name)
    raise AttributeError(name)
