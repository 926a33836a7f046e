"""Render parameters of the oracle.

The paper states only that the default parameters of 3D GS are used (Sec. 4.1.1);
each value here is a reading of that, listed with its reason in the design notes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass


@dataclass
class RenderParams:
    lowpass: float = 0.3          # px^2 added to the 2x2 screen covariance (also used for the plane)
    alpha_min: float = 1.0 / 255  # a splat whose alpha is below this is skipped at a pixel
    alpha_max: float = 0.99       # alpha is clamped to this (keeps 1/(1-alpha) bounded)
    T_min: float = 1e-4           # compositing stops before a splat would take T below this
    median_T: float = 0.5         # median depth: first splat whose transmittance after it is <= this
    clamp_margin: float = 0.15    # x/z, y/z inside J are clamped to the image widened by this fraction
    tile_w: int = 16
    tile_h: int = 16

    def ext_constant_f32(self) -> float:
        """2 ln(1/alpha_min), computed in double and rounded to float32.  The
        rectangle half-width sqrt(C * A_kk) bounds the ellipse alpha >= alpha_min
        for every opacity <= 1."""
        import numpy as np
        return float(np.float32(2.0 * math.log(1.0 / self.alpha_min)))


def clamp_limits_f32(width, height, fx, fy, cx, cy, margin):
    """Bounds of x/z and y/z used inside the Jacobian (image widened by ``margin``
    of its size on each side), computed in double and rounded to float32."""
    import numpy as np
    f32 = np.float32
    fx, fy, cx, cy = float(f32(fx)), float(f32(fy)), float(f32(cx)), float(f32(cy))
    mw, mh = margin * width, margin * height
    return (float(f32(-(cx + mw) / fx)), float(f32((width + mw - cx) / fx)),
            float(f32(-(cy + mh) / fy)), float(f32((height + mh - cy) / fy)))
