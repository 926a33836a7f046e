"""Per-pixel front-to-back compositing in FP64 (Eq. 3, Eq. 4, Sec. 1, Eq. 22).

For every pixel, the oracle gathers every Gaussian whose FP32 pixel rectangle
covers the pixel, sorts them by (depth-key bits, id) -- the order 3D GS uses and
the paper keeps (Sec. 3.1) -- and blends them one after another:

    Delta = (u_c - u, v_c - v)              pixel centre (i + 0.5, j + 0.5)
    sigma = 1/2 Delta^T conic Delta         (Eq. 1 with the 3D GS factor 1/2)
    alpha = min(alpha_max, o exp(-sigma))   skipped if alpha < alpha_min
    T'    = T (1 - alpha)                   stop before any splat with T' < T_min
    w     = alpha T                         blending weight omega_i (Eq. 3, 23)
    C    += w rgb,   N += w n               colour (Eq. 3), normal map (Sec. 1, Eq. 22)
    depth = z_c + p Delta of the first splat with T' <= median_T (Eq. 4, median, Sec. 1),
            else of the last contributor, else 0
    alpha map = 1 - T_final.

The per-pixel lists are padded to a rectangle so that the products over the list
are a plain ``cumprod``; every splat after the stop point gets alpha = 0.
Gradients come from torch autograd in FP64.

Each decision that FP32 could take the other way (alpha vs alpha_min, T' vs T_min,
T' vs median_T) is recorded with its relative margin so that tests can set
aside the pixels where FP32 and FP64 may legitimately differ.
"""
from __future__ import annotations

import numpy as np
import torch

from .params import RenderParams

DT = torch.float64


def candidate_pairs(dec, width, height, pixels=None):
    """(pixel, gaussian) pairs with the pixel inside the Gaussian's FP32 rect,
    sorted by (pixel, depth key, id).  ``pixels`` restricts to a set of flat
    pixel indices (row-major)."""
    ids = np.nonzero(dec["valid"])[0]
    rect = dec["rect"][ids]
    if pixels is not None:
        pixels = np.asarray(pixels, np.int64)
        px, py = pixels % width, pixels // width
        bx0, bx1, by0, by1 = px.min(), px.max(), py.min(), py.max()
        keep = (rect[:, 1] >= bx0) & (rect[:, 0] <= bx1) & (rect[:, 3] >= by0) & (rect[:, 2] <= by1)
        ids, rect = ids[keep], rect[keep].copy()
        rect[:, 0] = np.maximum(rect[:, 0], bx0)
        rect[:, 1] = np.minimum(rect[:, 1], bx1)
        rect[:, 2] = np.maximum(rect[:, 2], by0)
        rect[:, 3] = np.minimum(rect[:, 3], by1)
        mask = np.zeros(width * height, bool)
        mask[pixels] = True
    nx = rect[:, 1] - rect[:, 0] + 1
    ny = rect[:, 3] - rect[:, 2] + 1
    cnt = nx * ny
    g = np.repeat(ids, cnt)
    start = np.repeat(np.cumsum(cnt) - cnt, cnt)
    k = np.arange(int(cnt.sum()), dtype=np.int64) - start
    nxr = np.repeat(nx, cnt)
    pix = (np.repeat(rect[:, 2], cnt) + k // nxr) * width + np.repeat(rect[:, 0], cnt) + k % nxr
    if pixels is not None:
        sel = mask[pix]
        pix, g = pix[sel], g[sel]
    order = np.lexsort((g, dec["zkey"][g], pix))
    return pix[order], g[order]


def composite(pre, dec, width, height, params: RenderParams, pixels=None):
    """Render the selected pixels.  Returns dict of torch tensors (differentiable
    w.r.t. the entries of ``pre``): color (P,3), alpha (P,), depth (P,),
    normal (P,3), plus numpy diagnostics: pixels, n_contrib, last_pos,
    median_pos, margin (min relative margin of the discrete decisions)."""
    if pixels is None:
        pixels = np.arange(width * height, dtype=np.int64)
    pixels = np.asarray(pixels, np.int64)
    pix, g = candidate_pairs(dec, width, height, pixels)
    # map each pair to the row of its pixel in ``pixels``
    order = np.argsort(pixels, kind="stable")
    spix = pixels[order]
    row_sorted = np.searchsorted(spix, pix)
    row = order[row_sorted]
    P = len(pixels)
    counts = np.bincount(row, minlength=P)
    # padded layout: slot = position within the pixel's list; a stable regroup by
    # row keeps each pixel's (depth key, id) order
    perm = np.argsort(row, kind="stable")
    row_p, g_p = row[perm], g[perm]
    starts = np.cumsum(counts) - counts
    slot = np.arange(len(row_p)) - starts[row_p]
    K = int(counts.max()) if P and len(row_p) else 1
    K = max(K, 1)

    gidx = np.full((P, K), -1, np.int64)
    gidx[row_p, slot] = g_p
    valid = gidx >= 0
    pad = int(g_p[0]) if len(g_p) else 0   # any candidate: padded slots are masked out
    gsafe = torch.from_numpy(np.where(valid, gidx, pad))
    vmask = torch.from_numpy(valid)

    px = torch.from_numpy((pixels % width).astype(np.float64) + 0.5).to(DT)
    py = torch.from_numpy((pixels // width).astype(np.float64) + 0.5).to(DT)

    u = pre["u"][gsafe]
    v = pre["v"][gsafe]
    du = u - px[:, None]
    dv = v - py[:, None]
    ca = pre["conic"][:, 0][gsafe]
    cb = pre["conic"][:, 1][gsafe]
    cc = pre["conic"][:, 2][gsafe]
    sigma = 0.5 * (ca * du * du + cc * dv * dv) + cb * du * dv
    o = pre["opacity"][gsafe]
    alpha_raw = o * torch.exp(-sigma)
    alpha = torch.clamp(alpha_raw, max=params.alpha_max)

    with torch.no_grad():
        keep = vmask & (alpha >= params.alpha_min)
        a_eff = torch.where(keep, alpha, torch.zeros_like(alpha))
        T_incl = torch.cumprod(1.0 - a_eff, dim=1)
        included = keep & (T_incl >= params.T_min)
        # margins of the decisions up to (and including) the first stop
        T_prev = torch.cat([torch.ones_like(T_incl[:, :1]), T_incl[:, :-1]], dim=1)
        reached = vmask & (T_prev >= params.T_min)
        m_alpha = torch.where(reached, (alpha - params.alpha_min).abs() / params.alpha_min,
                              torch.full_like(alpha, np.inf))
        m_T = torch.where(reached & keep, (T_incl - params.T_min).abs() / params.T_min,
                          torch.full_like(alpha, np.inf))
        m_med = torch.where(included, (T_incl - params.median_T).abs() / params.median_T,
                            torch.full_like(alpha, np.inf))

    a_fin = torch.where(included, alpha, torch.zeros_like(alpha))
    one_minus = 1.0 - a_fin
    T_after = torch.cumprod(one_minus, dim=1)
    T_before = torch.cat([torch.ones_like(T_after[:, :1]), T_after[:, :-1]], dim=1)
    w = a_fin * T_before
    rgb = pre["rgb"][gsafe]
    nrm = pre["n"][gsafe]
    color = (w[..., None] * rgb).sum(dim=1)
    normal = (w[..., None] * nrm).sum(dim=1)
    T_final = T_after[:, -1]
    alpha_map = 1.0 - T_final

    with torch.no_grad():
        n_contrib = included.sum(dim=1)
        cross = included & (T_after <= params.median_T)
        has_cross = cross.any(dim=1)
        first_cross = torch.argmax(cross.to(torch.int8), dim=1)
        idxs = torch.arange(K).expand(P, K)
        last_pos = torch.where(included, idxs, torch.full_like(idxs, -1)).max(dim=1).values
        med_pos = torch.where(has_cross, first_cross, last_pos)
        # a median decision is ambiguous only up to the chosen splat
        upto = idxs <= med_pos[:, None].clamp(min=0)
        m_med = torch.where(upto, m_med, torch.full_like(m_med, np.inf))
        margin = torch.minimum(torch.minimum(m_alpha.min(dim=1).values, m_T.min(dim=1).values),
                               m_med.min(dim=1).values)
    ms = med_pos.clamp(min=0)
    z = pre["z"][gsafe]
    pp = pre["p"][gsafe]
    d_all = z + pp[..., 0] * du + pp[..., 1] * dv       # Eq. 4 at every candidate
    d_med = d_all.gather(1, ms[:, None]).squeeze(1)
    depth = torch.where(med_pos >= 0, d_med, torch.zeros_like(d_med))
    return dict(color=color, alpha=alpha_map, depth=depth, normal=normal,
                weights=w, gidx=gidx, d_all=d_all, T_final=T_final,
                pixels=pixels, n_contrib=n_contrib.numpy(), last_pos=last_pos.numpy(),
                median_pos=med_pos.numpy(), margin=margin.numpy(), K=K)
