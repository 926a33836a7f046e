"""The Mip-Splatting 3D smoothing filter that RaDe-GS adds to its Gaussians
(Sec. 4.1.1), in FP64 (test infrastructure only).

Each Gaussian k carries a filter variance v_k.  Its covariance becomes
Sigma + v_k I and its opacity is scaled by sqrt(det Sigma / det(Sigma + v_k I)),
which keeps the integral of the opacity-weighted Gaussian unchanged.  Since
Sigma = R S S^T R^T, adding v_k I keeps R and replaces every scale s_i by
s~_i = sqrt(s_i^2 + v_k); the opacity factor is prod_i s_i / s~_i.

v_k comes from the cameras: with nu_k the largest sampling rate f_n / z_n over
the views n in which the centre lies in front (z_n > near) and projects inside
the image widened by 15 % on each side, v_k = c / nu_k^2 = c min_n (z_n / f_n)^2
with c = 0.2 (Mip-Splatting's default).  A Gaussian seen by no view gets the
largest v of the seen ones (0 if none is seen).  f_n is the view's fx.
"""
from __future__ import annotations

import numpy as np
import torch

F = np.float32


def apply_filter(scales: torch.Tensor, opacities: torch.Tensor, var: torch.Tensor):
    """FP64, differentiable: (s~, o') from (s, o) and the filter variances."""
    st = torch.sqrt(scales * scales + var[:, None])
    return st, opacities * torch.prod(scales / st, dim=1)


def apply_filter_f32(scales: np.ndarray, opacities: np.ndarray, var: np.ndarray):
    """The same in FP32 with a fixed operation order (each step rounded):
    s~ = sqrt(s*s + v); o' = ((o * (s0/s~0)) * (s1/s~1)) * (s2/s~2).  The binning
    decisions are taken on these values."""
    s = np.asarray(scales, F)
    o = np.asarray(opacities, F)
    v = np.asarray(var, F)
    with np.errstate(all="ignore"):
        st = np.sqrt(s * s + v[:, None])
        r = s / st
        op = ((o * r[:, 0]) * r[:, 1]) * r[:, 2]
    return st.astype(F), op.astype(F)


def filter_variance(means, cams, scale: float = 0.2, margin: float = 0.15, near: float = None):
    """v_k for every Gaussian from the views ``cams`` (FP64).  Returns (v, seen)."""
    m = np.asarray(means, np.float64)
    best = np.full(len(m), np.inf)
    for cam in cams:
        V = np.asarray(cam.viewmat, np.float64)
        xc = m @ V[:3, :3].T + V[:3, 3]
        z = xc[:, 2]
        zn = cam.near if near is None else near
        with np.errstate(all="ignore"):
            u = cam.fx * xc[:, 0] / z + cam.cx
            v = cam.fy * xc[:, 1] / z + cam.cy
        inside = ((z > zn) & (u >= -margin * cam.width) & (u <= (1 + margin) * cam.width)
                  & (v >= -margin * cam.height) & (v <= (1 + margin) * cam.height))
        r = np.where(inside, (z / cam.fx) ** 2, np.inf)
        best = np.minimum(best, r)
    seen = np.isfinite(best)
    out = scale * best
    fill = out[seen].max() if seen.any() else 0.0
    out[~seen] = fill
    return out, seen
