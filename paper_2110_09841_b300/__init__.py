"""Cutting voxel projector (Kulvait & Rose, arXiv 2110.09841) for NVIDIA B300.

    from paper_2110_09841_b300 import Projector, inputs
    geom = inputs.workload_geometry("cvp32")
    A = Projector(geom, variant="exact", scaling="cos")
    b = A.project(x)          # x: float32 CUDA tensor [nz, ny, nx]
    xt = A.backproject(b)     # float32 CUDA tensor [nz, ny, nx]

Also: A.project_batch / A.backproject_batch (one launch per batch), A.cgls (CGLS on the
device), A.autotune (forward tile choice), A.siddon (ray-driven comparator); autograd.project /
autograd.backproject (differentiable operator); conv, unet and warmstart (tensor-core 3D
convolutions and the U-Net warm start for CGLS).

The compute runs in libkct.so and libkct_conv.so (hand-written CUDA for sm_103a); this
package only marshals arguments. There is no CPU fallback.
"""
from . import inputs  # noqa: F401

__all__ = ["Projector", "KctError", "inputs"]


def __getattr__(name):
    if name in ("Projector", "KctError"):
        from . import kct

        return getattr(kct, name)
    raise AttributeError(name)
