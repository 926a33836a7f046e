"""Oracle entry points: forward maps and FP64 gradients for one camera."""
from __future__ import annotations

import numpy as np
import torch

from . import binning, composite as comp, filter3d, gaussians
from .params import RenderParams

DT = torch.float64
PARAM_NAMES = ("means", "scales", "quats", "opacities", "sh")
PRE2D = ("u", "v", "conic", "opacity", "rgb", "n", "z", "p")


def _leaves(scene, requires_grad):
    out = {}
    for k in PARAM_NAMES:
        # float32 inputs are promoted exactly; float64 inputs (finite differences) are kept
        a = np.asarray(getattr(scene, k)).astype(np.float64)
        out[k] = torch.tensor(a, dtype=DT, requires_grad=requires_grad)
    return out


def _project(leaves, scene, cam, params, route="schur"):
    scales, opacities = leaves["scales"], leaves["opacities"]
    fv = getattr(scene, "filter_var", None)
    if fv is not None:   # Mip-Splatting 3D filter (Sec. 4.1.1)
        scales, opacities = filter3d.apply_filter(scales, opacities,
                                                  torch.tensor(np.asarray(fv, np.float64), dtype=DT))
    return gaussians.project(leaves["means"], scales, leaves["quats"], opacities, leaves["sh"],
                             scene.sh_degree, cam, params, route=route)


def _chunks(pixels, size):
    for i in range(0, len(pixels), size):
        yield pixels[i:i + size]


def render(scene, cam, params: RenderParams = None, pixels=None, chunk=4096, route="schur"):
    """Forward maps in FP64 for the selected flat pixel indices (default: all).

    Returns a dict of numpy arrays: color (P,3), alpha, depth, normal (P,3),
    margin, n_contrib, pixels, plus the FP32 binning decisions ``dec``."""
    params = params or RenderParams()
    dec = binning.decide_scene(scene, cam, params)
    with torch.no_grad():
        pre = _project(_leaves(scene, False), scene, cam, params, route)
        if pixels is None:
            pixels = np.arange(cam.width * cam.height, dtype=np.int64)
        pixels = np.asarray(pixels, np.int64)
        outs = {k: [] for k in ("color", "alpha", "depth", "normal", "margin", "n_contrib")}
        for px in _chunks(pixels, chunk):
            r = comp.composite(pre, dec, cam.width, cam.height, params, px)
            for k in ("color", "alpha", "depth", "normal"):
                outs[k].append(r[k].numpy())
            outs["margin"].append(r["margin"])
            outs["n_contrib"].append(r["n_contrib"])
    res = {k: np.concatenate(v) for k, v in outs.items()}
    res["pixels"] = pixels
    res["dec"] = dec
    res["pre"] = {k: pre[k].numpy() for k in PRE2D}
    return res


def render_grads(scene, cam, upstream, params: RenderParams = None, pixels=None, chunk=4096,
                 route="schur"):
    """FP64 gradients of L = sum(dC*color) + sum(dA*alpha) + sum(dD*depth) + sum(dN*normal).

    ``upstream`` = (dcolor (3,H,W), dalpha (H,W), ddepth (H,W), dnormal (3,H,W)).
    Only the selected pixels contribute.  Returns (param_grads, grads2d, maps):
    param_grads has means, scales, quats, opacities, sh; grads2d has the
    gradients w.r.t. the per-Gaussian 2D quantities u, v, conic(a,b,c), opacity,
    rgb, n, z, p (the quantities the compositing stage reads)."""
    params = params or RenderParams()
    dC, dA, dD, dN = [np.asarray(x, np.float64) for x in upstream]
    W_, H_ = cam.width, cam.height
    dC = dC.reshape(3, H_ * W_)
    dN = dN.reshape(3, H_ * W_)
    dA = dA.reshape(H_ * W_)
    dD = dD.reshape(H_ * W_)
    dec = binning.decide_scene(scene, cam, params)
    leaves = _leaves(scene, True)
    pre = _project(leaves, scene, cam, params, route)
    # detached copies of the 2D quantities: the composite is differentiated
    # chunk by chunk w.r.t. these, then the sum is pushed through the projection.
    pre_d = {k: pre[k].detach().clone().requires_grad_(True) for k in PRE2D}
    acc = {k: torch.zeros_like(pre_d[k]) for k in PRE2D}
    if pixels is None:
        pixels = np.arange(W_ * H_, dtype=np.int64)
    pixels = np.asarray(pixels, np.int64)
    maps = {k: [] for k in ("color", "alpha", "depth", "normal", "margin")}
    for px in _chunks(pixels, chunk):
        r = comp.composite(pre_d, dec, W_, H_, params, px)
        loss = ((r["color"] * torch.from_numpy(dC[:, px].T)).sum()
                + (r["alpha"] * torch.from_numpy(dA[px])).sum()
                + (r["depth"] * torch.from_numpy(dD[px])).sum()
                + (r["normal"] * torch.from_numpy(dN[:, px].T)).sum())
        gs = torch.autograd.grad(loss, [pre_d[k] for k in PRE2D], allow_unused=True)
        for k, gk in zip(PRE2D, gs):
            if gk is not None:
                acc[k] += gk
        for k in ("color", "alpha", "depth", "normal"):
            maps[k].append(r[k].detach().numpy())
        maps["margin"].append(r["margin"])
    vm = torch.from_numpy(dec["valid"])
    total = sum((pre[k][vm] * acc[k][vm]).sum() for k in PRE2D)
    pg = torch.autograd.grad(total, [leaves[k] for k in PARAM_NAMES], allow_unused=True)
    param_grads = {k: (g.numpy() if g is not None else np.zeros_like(leaves[k].detach().numpy()))
                   for k, g in zip(PARAM_NAMES, pg)}
    grads2d = {k: acc[k].numpy() for k in PRE2D}
    maps = {k: np.concatenate(v) for k, v in maps.items()}
    maps["pixels"] = pixels
    maps["dec"] = dec
    return param_grads, grads2d, maps
