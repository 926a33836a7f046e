"""Depth distortion (Eq. 23) and normal consistency (Eq. 24) in FP64.

* Eq. 23: L_d = sum_{i,j} w_i w_j (d_i - d_j)^2 per pixel, over the splats that
  blend at the pixel, with d_i the planar depth of splat i there (Eq. 4) and
  the weights w detached (Sec. 4.1.1).  Written as the plain double sum.
* Eq. 24: L_n = sum_i w_i (1 - n_i^T n~) per pixel, with n~ the normal of the
  rendered (median) depth map by finite differences: the depth map is
  back-projected to camera space, P(i, j) = D(i, j) r(i, j) with
  r = ((i + 1/2 - cx)/fx, (j + 1/2 - cy)/fy, 1), and
  n~ = normalize((P(i, j+1) - P(i, j-1)) x (P(i+1, j) - P(i-1, j))),
  which points toward the camera.  Reading (the paper does not say): n~ is
  defined on interior pixels whose 4-neighbourhood and centre all have a
  non-zero alpha; elsewhere L_n is 0.  Gradients flow through w, n_i and n~.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binning, composite as comp
from .params import RenderParams
from .render import PARAM_NAMES, PRE2D, _leaves, _project

DT = torch.float64


def depth_distortion_pairwise(weights: torch.Tensor, d_all: torch.Tensor, chunk: int = 256) -> torch.Tensor:
    """Eq. 23 per pixel as the plain double sum over splat pairs (no gradient)."""
    out = []
    with torch.no_grad():
        for i in range(0, weights.shape[0], chunk):
            w, d = weights[i:i + chunk], d_all[i:i + chunk]
            diff = d[:, :, None] - d[:, None, :]
            out.append((w[:, :, None] * w[:, None, :] * diff * diff).sum(dim=(1, 2)))
    return torch.cat(out) if out else torch.zeros(0, dtype=DT)


def depth_distortion(weights: torch.Tensor, d_all: torch.Tensor) -> torch.Tensor:
    """Eq. 23 per pixel, weights detached, through the expansion of the square:
    sum_ij w_i w_j (d_i - d_j)^2 = 2 (W S2 - S1^2), W = sum w, S1 = sum w d,
    S2 = sum w d^2 (the tests check it against the double sum)."""
    w = weights.detach()
    W = w.sum(dim=1)
    S1 = (w * d_all).sum(dim=1)
    S2 = (w * d_all * d_all).sum(dim=1)
    return 2.0 * (W * S2 - S1 * S1)


def depth_normals(depth: torch.Tensor, alpha: torch.Tensor, cam):
    """(H, W) depth and alpha -> (H, W, 3) normals of the back-projected depth
    map and the (H, W) mask of pixels where they are defined."""
    H, W = depth.shape
    f32 = lambda x: float(np.float32(x))
    fx, fy, cx, cy = f32(cam.fx), f32(cam.fy), f32(cam.cx), f32(cam.cy)
    ii = torch.arange(W, dtype=DT) + 0.5
    jj = torch.arange(H, dtype=DT) + 0.5
    rx = ((ii - cx) / fx)[None, :].expand(H, W)
    ry = ((jj - cy) / fy)[:, None].expand(H, W)
    P = torch.stack([depth * rx, depth * ry, depth], dim=-1)
    n = torch.zeros(H, W, 3, dtype=DT)
    ok = torch.zeros(H, W, dtype=torch.bool)
    if H < 3 or W < 3:
        return n, ok
    a = P[1:-1, 2:] - P[1:-1, :-2]          # along +x (columns)
    b = P[2:, 1:-1] - P[:-2, 1:-1]          # along +y (rows)
    c = torch.cross(b, a, dim=-1)
    nrm = c.norm(dim=-1)
    alive = alpha > 0
    inner = (alive[1:-1, 1:-1] & alive[1:-1, 2:] & alive[1:-1, :-2] & alive[2:, 1:-1] & alive[:-2, 1:-1]
             & (nrm.detach() > 0))
    safe = torch.where(inner, nrm, torch.ones_like(nrm))
    nt = torch.where(inner[..., None], c / safe[..., None], torch.zeros_like(c))
    n = torch.zeros(H, W, 3, dtype=DT)
    n = n.index_put((torch.arange(1, H - 1)[:, None], torch.arange(1, W - 1)[None, :]), nt)
    ok[1:-1, 1:-1] = inner
    return n, ok


def normal_consistency(weights: torch.Tensor, n_splat: torch.Tensor, n_tilde: torch.Tensor,
                       ok: torch.Tensor) -> torch.Tensor:
    """Eq. 24 per pixel: sum_i w_i (1 - n_i^T n~), zero where n~ is undefined."""
    dot = (n_splat * n_tilde[:, None, :]).sum(dim=-1)
    Ln = (weights * (1.0 - dot)).sum(dim=1)
    return torch.where(ok, Ln, torch.zeros_like(Ln))


def render_with_losses(scene, cam, upstream=None, params: RenderParams = None):
    """Whole-image forward with both losses; with ``upstream`` also FP64 gradients.

    ``upstream`` = (dcolor (3,H,W), dalpha, ddepth, dnormal (3,H,W), ddist, dnloss)
    weights the six maps; returns (maps, param_grads, grads2d), the last two None
    without ``upstream``.  Small images only (one dense autograd graph)."""
    params = params or RenderParams()
    H, W = cam.height, cam.width
    dec = binning.decide_scene(scene, cam, params)
    leaves = _leaves(scene, upstream is not None)
    pre = _project(leaves, scene, cam, params)
    pre_d = {k: pre[k].detach().clone().requires_grad_(upstream is not None) for k in PRE2D}
    pix = np.arange(H * W, dtype=np.int64)
    r = comp.composite(pre_d, dec, W, H, params, pix)
    Ld = depth_distortion(r["weights"], r["d_all"])
    depth = r["depth"].reshape(H, W)
    alpha = r["alpha"].reshape(H, W)
    nt, ok = depth_normals(depth, alpha.detach(), cam)
    gidx = torch.from_numpy(np.where(r["gidx"] >= 0, r["gidx"], 0))
    n_splat = pre_d["n"][gidx]
    Ln = normal_consistency(r["weights"], n_splat, nt.reshape(-1, 3), ok.reshape(-1))
    maps = dict(color=r["color"], alpha=r["alpha"], depth=r["depth"], normal=r["normal"], dist=Ld,
                nloss=Ln, margin=r["margin"], n_tilde=nt.reshape(-1, 3), n_ok=ok.reshape(-1),
                weights=r["weights"], d_all=r["d_all"])
    if upstream is None:
        return {k: (v.detach().numpy() if torch.is_tensor(v) else v) for k, v in maps.items()}, None, None
    dC, dA, dD, dN, dLd, dLn = [torch.from_numpy(np.asarray(x, np.float64)).to(DT) for x in upstream]
    loss = ((r["color"] * dC.reshape(3, -1).T).sum() + (r["alpha"] * dA.reshape(-1)).sum()
            + (r["depth"] * dD.reshape(-1)).sum() + (r["normal"] * dN.reshape(3, -1).T).sum()
            + (Ld * dLd.reshape(-1)).sum() + (Ln * dLn.reshape(-1)).sum())
    gs = torch.autograd.grad(loss, [pre_d[k] for k in PRE2D], allow_unused=True)
    acc = {k: (g if g is not None else torch.zeros_like(pre_d[k])) for k, g in zip(PRE2D, gs)}
    vm = torch.from_numpy(dec["valid"])
    total = sum((pre[k][vm] * acc[k][vm]).sum() for k in PRE2D)
    pg = torch.autograd.grad(total, [leaves[k] for k in PARAM_NAMES], allow_unused=True)
    param_grads = {k: (g.numpy() if g is not None else np.zeros(leaves[k].shape)) for k, g in zip(PARAM_NAMES, pg)}
    maps_np = {k: (v.detach().numpy() if torch.is_tensor(v) else v) for k, v in maps.items()}
    return maps_np, param_grads, {k: acc[k].numpy() for k in PRE2D}
