"""Oracle entry points: forward maps and FP64 gradients for one camera."""
from __future__ import annotations

import contextlib
import sys

import numpy as np
import torch

from . import binning, composite as comp, filter3d, gaussians
from .params import RenderParams

DT = torch.float64
PARAM_NAMES = ("means", "scales", "quats", "opacities", "sh")
PRE2D = ("u", "v", "conic", "opacity", "rgb", "n", "z", "p")


@contextlib.contextmanager
def evaluated_in(dtype):
    """Runs the oracle's floating-point arithmetic in ``dtype`` instead of FP64.

    A test instrument only: the FP64 results are the reference.  The same
    definition evaluated in FP32 shows how far FP32 rounding alone moves each
    result, which is the scale against which an FP32 implementation's
    differences from the FP64 values are weighed entry by entry.  The binning
    decisions are FP32 either way."""
    from . import appearance, losses
    mods = (gaussians, comp, losses, appearance, sys.modules[__name__])
    old = [m.DT for m in mods]
    try:
        for m in mods:
            m.DT = dtype
        yield
    finally:
        for m, d in zip(mods, old):
            m.DT = d


def fp32_spread(grad_fn, scene, samples=4, seed=0):
    """FP64 gradients and, entry by entry, how far FP32 evaluations move them.

    A test instrument (no counterpart in the paper).  ``grad_fn(scene)`` returns
    a dict of gradient arrays computed by the oracle.  It is evaluated once in
    FP64 (the reference) and ``samples`` times in FP32: at the scene's own
    parameters, then at parameters each moved by -1, 0 or +1 unit in the last
    place of FP32, at random.  Returns (ref, spread), spread holding the
    largest |FP32 - FP64| of each entry over the samples: the amount by which
    rounding to FP32 inside the computation, or a one-ulp change of an input,
    moves that entry.  It is large only where the entry is ill-conditioned
    (terms that cancel over the pixels, thin splats whose conic inverts a
    nearly singular 2x2 matrix), and an FP32 implementation cannot be asked to
    match the FP64 value more closely than a small multiple of it."""
    ref = {k: np.asarray(v, np.float64) for k, v in grad_fn(scene).items()}
    spread = {k: np.zeros_like(v) for k, v in ref.items()}
    rng = np.random.default_rng(seed)
    for s in range(samples):
        sc = scene
        if s > 0:
            moved = {}
            for k in PARAM_NAMES:
                a = np.ascontiguousarray(getattr(scene, k), np.float32)
                moved[k] = (a.view(np.int32) + rng.integers(-1, 2, a.shape).astype(np.int32)).view(np.float32)
            sc = type(scene)(**{**scene.__dict__, **moved})
        with evaluated_in(torch.float32):
            g = grad_fn(sc)
        for k in ref:
            spread[k] = np.maximum(spread[k], np.abs(np.asarray(g[k], np.float64) - ref[k]))
    return ref, spread


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
        t = lambda a: torch.from_numpy(a).to(DT)
        loss = ((r["color"] * t(dC[:, px].T)).sum() + (r["alpha"] * t(dA[px])).sum()
                + (r["depth"] * t(dD[px])).sum() + (r["normal"] * t(dN[:, px].T)).sum())
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

