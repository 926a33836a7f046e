"""Plain, slow FP64 CPU oracle for the RaDe-GS rasterizer (arxiv 2406.01467).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use it.  It shares no code with the CUDA library; the two meet only
in the seeded input arrays.

Layout
------
``params``     render parameters the paper leaves to the 3D GS defaults (Sec. 4.1.1).
``sh``         real spherical harmonics from their definition (colour, Eq. 3's c_i).
``gaussians``  per-Gaussian quantities in FP64 torch ops: Eq. 1-2 (EWA projection),
               Eq. 8-15 (ray-space intersection, depth plane p, two independent
               routes), Eq. 18-22 (ray-space plane normal and camera-space normal).
``binning``    the tile lists and their sort order, decided in FP32 exactly as
               specified (pixel rectangles, (tile, depth, id) order).
``composite``  per-pixel front-to-back alpha blending (Eq. 3) of colour, alpha,
               planar depth (Eq. 4) and normal, with the median depth (Sec. 1);
               gradients by torch autograd in FP64.
``losses``     depth distortion (Eq. 23, weights detached) and normal consistency
               (Eq. 24, normals of the depth map by central differences).
``filter3d``   the Mip-Splatting 3D filter (Sigma + v I with opacity compensation)
               and its per-Gaussian variance from the cameras (Sec. 4.1.1).
``appearance`` decoupled per-view appearance (Sec. 4.1.1): embedding -> MLP ->
               colour affine, L1 loss, Adam.

Parity pins: every function is checked against a value the paper or
mathematics fixes (closed forms, library routines, invariants, brute force,
finite differences) by the ``-m "not gpu"`` tests.
"""
from .params import RenderParams  # noqa: F401
from . import sh, gaussians, binning, composite, losses, filter3d, appearance  # noqa: F401
from .render import evaluated_in, fp32_spread, render, render_grads  # noqa: F401
