"""Cutting voxel projector (Kulvait & Rose, arXiv 2110.09841) for NVIDIA B300.

    from paper_2110_09841_b300 import Projector, inputs
    geom = inputs.workload_geometry("cvp32")
    A = Projector(geom, variant="exact", scaling="cos")
    b = A.project(x)          # x: float32 CUDA tensor [nz, ny, nx]
    xt = A.backproject(b)     # float32 CUDA tensor [nz, ny, nx]

The compute runs in libkct.so (hand-written CUDA for sm_103a); this package only
marshals arguments. There is no CPU fallback.
"""
from . import inputs  # noqa: F401

__all__ = ["Projector", "KctError", "inputs"]


def __getattr__(name):
    if name in ("Projector", "KctError"):
        from . import kct

        return getattr(kct, name)
    raise AttributeError(name)
