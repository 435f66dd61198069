"""GB300-native (sm_103a) SBR-on-points path of PointEMRay (arXiv 2408.15583).

The compute lives in ``libpointemray.so`` (CUDA kernels behind the C ABI of
``include/pointemray.h``); ``paper_2408_15583_gb300.api`` holds thin
torch-facing wrappers and ``build`` compiles the library in-tree.
"""
from .build import build  # noqa: F401

__all__ = ["build"]
