"""GB300-native differentiable 3D Gaussian-splatting rasterizer (forward and backward, with SE(3)
pose gradients), the hot path of every tracking and mapping iteration of RGS-SLAM.

The compute path is the sm_103a CUDA library ``librgs.so`` behind a C ABI (``include/rgs.h``);
``paper_2601_00705_gb300.binding`` marshals arguments to it and ``paper_2601_00705_gb300.render``
wraps it in a ``torch.autograd.Function``. Submodules are imported lazily so that the seeded
input generators in ``synthetic`` load without a GPU.
"""
__all__ = ["synthetic", "binding", "render", "build"]
