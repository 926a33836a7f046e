"""Tile lists and compositing order, decided in FP32.

Which Gaussians a pixel sees, and in which order, are integer decisions taken in
floating point, so the oracle takes them in the kernel's precision: FP32, every
operation correctly rounded and performed one at a time in the order below
(numpy float32 arithmetic never fuses a multiply and an add).  The paper does
not describe binning; it inherits it from 3D GS (Sec. 4.1.1).  The order is:

 1. x_c = ((R0 m_x + R1 m_y) + R2 m_z) + t, row by row; z = x_c[2]; invalid unless z > near.
 2. iz = 1/z; tx = x iz; ty = y iz; u = fx tx + cx; v = fy ty + cy.
 3. quaternion: n2 = ((w w + x x) + y y) + z z, invalid unless n2 > 0; r = 1/sqrt(n2);
    (w, x, y, z) *= r; rotation entries from the products xx, yy, ... (Eq. 1's R).
 4. M = R_q diag(s); J rows 1-2 (Eq. 2): j00 = fx iz, j02 = -(fx clamp(tx)) iz,
    j11 = fy iz, j12 = -(fy clamp(ty)) iz.
 5. T = J[0:2] W: T0k = j00 W0k + j02 W2k, T1k = j11 W1k + j12 W2k.
 6. G_ik = ((T_i0 M_0k + T_i1 M_1k) + T_i2 M_2k) for i in {0,1}.
 7. A00 = ((G00 G00 + G01 G01) + G02 G02) + lowpass; A11 likewise (Eq. 2's 2x2 block).
 8. ex = sqrt(C A00), ey = sqrt(C A11), C = float32(2 ln(1/alpha_min)): the
    axis-aligned box of the ellipse on which alpha = alpha_min for opacity 1.
 9. xlo = (u - ex) - 0.5, xhi = (u + ex) - 0.5 (same for y); invalid unless
    xhi >= 0, xlo <= W-1, yhi >= 0, ylo <= H-1 and opacity >= alpha_min (a splat
    whose opacity is below alpha_min can never reach it, since alpha <= opacity).
10. pixel rect i0 = max(0, ceil xlo), i1 = min(W-1, floor xhi) (same for j);
    invalid if empty.  Tile rect = pixel rect // tile size.
11. sort key: (tile id, float bits of z, Gaussian id), ascending.
"""
from __future__ import annotations

import numpy as np

from . import filter3d
from .params import RenderParams, clamp_limits_f32

F = np.float32


def decide(means, scales, quats, opacities, cam, params: RenderParams, filter_var=None):
    """Per-Gaussian FP32 decisions: validity, depth key, pixel and tile rectangles.
    With ``filter_var`` the Mip-Splatting 3D filter is applied first (FP32 chain
    of ``filter3d.apply_filter_f32``)."""
    m = np.asarray(means, F)
    s = np.asarray(scales, F)
    qq = np.asarray(quats, F)
    o = np.asarray(opacities, F)
    if filter_var is not None:
        s, o = filter3d.apply_filter_f32(s, o, filter_var)
    V = np.asarray(cam.viewmat, F)
    fx, fy, cx, cy = F(cam.fx), F(cam.fy), F(cam.cx), F(cam.cy)
    W, H = int(cam.width), int(cam.height)
    lims = [F(x) for x in clamp_limits_f32(W, H, fx, fy, cx, cy, params.clamp_margin)]
    near = F(cam.near)
    lp = F(params.lowpass)
    C = F(params.ext_constant_f32())
    one, two, half = F(1), F(2), F(0.5)

    with np.errstate(all="ignore"):
        xc = [((V[i, 0] * m[:, 0] + V[i, 1] * m[:, 1]) + V[i, 2] * m[:, 2]) + V[i, 3] for i in range(3)]
        z = xc[2]
        valid = z > near
        iz = one / z
        tx = xc[0] * iz
        ty = xc[1] * iz
        u = fx * tx + cx
        v = fy * ty + cy

        qw, qx, qy, qz = qq[:, 0], qq[:, 1], qq[:, 2], qq[:, 3]
        n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz
        valid &= n2 > 0
        r = one / np.sqrt(n2)
        w, x, y, zq = qw * r, qx * r, qy * r, qz * r
        xx, yy, zz = x * x, y * y, zq * zq
        xy, xz, yz = x * y, x * zq, y * zq
        wx, wy, wz = w * x, w * y, w * zq
        Rq = [[one - two * (yy + zz), two * (xy - wz), two * (xz + wy)],
              [two * (xy + wz), one - two * (xx + zz), two * (yz - wx)],
              [two * (xz - wy), two * (yz + wx), one - two * (xx + yy)]]
        M = [[Rq[i][k] * s[:, k] for k in range(3)] for i in range(3)]

        txc = np.minimum(np.maximum(tx, lims[0]), lims[1])
        tyc = np.minimum(np.maximum(ty, lims[2]), lims[3])
        j00 = fx * iz
        j02 = -(fx * txc) * iz
        j11 = fy * iz
        j12 = -(fy * tyc) * iz
        T0 = [j00 * V[0, k] + j02 * V[2, k] for k in range(3)]
        T1 = [j11 * V[1, k] + j12 * V[2, k] for k in range(3)]
        G0 = [((T0[0] * M[0][k] + T0[1] * M[1][k]) + T0[2] * M[2][k]) for k in range(3)]
        G1 = [((T1[0] * M[0][k] + T1[1] * M[1][k]) + T1[2] * M[2][k]) for k in range(3)]
        A00 = ((G0[0] * G0[0] + G0[1] * G0[1]) + G0[2] * G0[2]) + lp
        A11 = ((G1[0] * G1[0] + G1[1] * G1[1]) + G1[2] * G1[2]) + lp
        ex = np.sqrt(C * A00)
        ey = np.sqrt(C * A11)
        xlo = (u - ex) - half
        xhi = (u + ex) - half
        ylo = (v - ey) - half
        yhi = (v + ey) - half
        valid &= (xhi >= 0) & (xlo <= F(W - 1)) & (yhi >= 0) & (ylo <= F(H - 1))
        valid &= o >= F(params.alpha_min)
        i0 = np.where(valid, np.maximum(F(0), np.ceil(xlo)), 0).astype(np.int64)
        i1 = np.where(valid, np.minimum(F(W - 1), np.floor(xhi)), -1).astype(np.int64)
        j0 = np.where(valid, np.maximum(F(0), np.ceil(ylo)), 0).astype(np.int64)
        j1 = np.where(valid, np.minimum(F(H - 1), np.floor(yhi)), -1).astype(np.int64)
    valid &= (i0 <= i1) & (j0 <= j1)
    tw, th = params.tile_w, params.tile_h
    tx0, tx1 = i0 // tw, i1 // tw
    ty0, ty1 = j0 // th, j1 // th
    touched = np.where(valid, (tx1 - tx0 + 1) * (ty1 - ty0 + 1), 0)
    zkey = z.astype(F).view(np.uint32)
    return dict(valid=valid, zkey=zkey, u=u, v=v, A00=A00, A11=A11,
                rect=np.stack([i0, i1, j0, j1], 1), tile_rect=np.stack([tx0, tx1, ty0, ty1], 1),
                tiles_touched=touched.astype(np.int64))


def tile_grid(cam, params: RenderParams):
    tiles_x = -(-int(cam.width) // params.tile_w)
    tiles_y = -(-int(cam.height) // params.tile_h)
    return tiles_x, tiles_y


def tile_lists(dec, cam, params: RenderParams, brute_force: bool = False):
    """Sorted (tile, Gaussian) pairs and per-tile ranges.

    ``brute_force`` tests every (Gaussian, tile) pair for rectangle overlap
    (small inputs only); otherwise each Gaussian's tile rectangle is enumerated.
    Order: tile id, then depth-key bits, then Gaussian id (np.lexsort)."""
    tiles_x, tiles_y = tile_grid(cam, params)
    T = tiles_x * tiles_y
    ids = np.nonzero(dec["valid"])[0]
    tr = dec["tile_rect"][ids]
    if brute_force:
        tix = np.arange(T) % tiles_x
        tiy = np.arange(T) // tiles_x
        hit = ((tix[None, :] >= tr[:, 0:1]) & (tix[None, :] <= tr[:, 1:2]) &
               (tiy[None, :] >= tr[:, 2:3]) & (tiy[None, :] <= tr[:, 3:4]))
        gi, ti = np.nonzero(hit)
        g = ids[gi]
        tile = ti
    else:
        nx = tr[:, 1] - tr[:, 0] + 1
        ny = tr[:, 3] - tr[:, 2] + 1
        cnt = nx * ny
        g = np.repeat(ids, cnt)
        start = np.repeat(np.cumsum(cnt) - cnt, cnt)
        k = np.arange(int(cnt.sum())) - start
        nxr = np.repeat(nx, cnt)
        tile = (np.repeat(tr[:, 2], cnt) + k // nxr) * tiles_x + np.repeat(tr[:, 0], cnt) + k % nxr
    order = np.lexsort((g, dec["zkey"][g], tile))
    tile = tile[order].astype(np.int64)
    g = g[order].astype(np.int64)
    ranges = np.zeros((T, 2), np.int64)
    if len(tile):
        first = np.searchsorted(tile, np.arange(T), side="left")
        last = np.searchsorted(tile, np.arange(T), side="right")
        ranges[:, 0], ranges[:, 1] = first, last
    return tile, g, ranges


def decide_scene(scene, cam, params: RenderParams):
    """``decide`` for a scene object (its 3D filter variances, if any, included)."""
    return decide(scene.means, scene.scales, scene.quats, scene.opacities, cam, params,
                  getattr(scene, "filter_var", None))
