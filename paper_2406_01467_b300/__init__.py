"""B300-native depth/normal Gaussian-splat rasterizer (RaDe-GS, arxiv 2406.01467).

The compute path is libgs.so (hand-written sm_103a CUDA behind the C ABI of
include/gs.h); this package holds its Python binding and the seeded synthetic
scene generators.  ``rasterize`` renders colour, alpha, median planar depth and
normal maps and is differentiable through the library's backward kernels.
"""
from .rasterize import Frame, RenderParams, SceneTensors, rasterize  # noqa: F401

__all__ = ["Frame", "RenderParams", "SceneTensors", "rasterize"]
