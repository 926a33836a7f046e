"""Parity of the depth-distortion (Eq. 23) and normal-consistency (Eq. 24) maps
and of their gradients with the FP64 oracle, through the C ABI.

Tolerances.  L_d: relative 1e-4 of the value plus 1e-4 of its sensitivity to
the planar depths (W sum_k w_k |d_k - mean| max|d|, from FP32 depths) and a
floor of 1e-7 W^2 max(d)^2.  L_n: the normal of the depth map divides depth
differences by |a| ~ 2 depth / f, so FP32 depth rounding is amplified by the
conditioning kappa = (|da|/|a| + |db|/|b|) / sin(a, b) with |da| = 1e-5
depth (1 + |r|); pixels with kappa > 1e-2 are excluded and the rest compared at
1e-4 + 4 |N| kappa.  The stencil alone is checked on the GPU's own maps at
1e-4.  Gradients: every entry within 1e-3 relative plus 16 times the change
FP32 evaluations of the oracle make to it (tests/_util.py), with the
upstream zeroed where a discrete decision of the pixel (or, for L_n, of its
stencil) is within the FP32/FP64 ambiguity margin or L_n is ill-conditioned.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import losses as olosses
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes
from tests._util import assert_grads_close, oracle_grads_with_spread, AMBIG_MARGIN, compare_maps, gpu_maps_at, grad2d_to_record, oracle_params

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _cam():
    # ragged in both directions for every tile size
    return scenes.Camera(np.eye(4), 128.0, 128.0, 62.5, 53.5, 125, 107)


def _frame(sc, cam, p):
    fr = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p)
    fr.forward()
    torch.cuda.synchronize()
    return fr


def _dilate(m):
    out = m.copy()
    out[1:] |= m[:-1]
    out[:-1] |= m[1:]
    out[:, 1:] |= m[:, :-1]
    out[:, :-1] |= m[:, 1:]
    return out


def _conditioning(depth, cam, rel=1e-5):
    """kappa of the depth-map normal at every pixel (inf where undefined)."""
    H, W = depth.shape
    rx = ((np.arange(W) + 0.5 - cam.cx) / cam.fx)[None, :].repeat(H, 0)
    ry = ((np.arange(H) + 0.5 - cam.cy) / cam.fy)[:, None].repeat(W, 1)
    P = np.stack([depth * rx, depth * ry, depth], -1)
    kap = np.full((H, W), np.inf)
    a = P[1:-1, 2:] - P[1:-1, :-2]
    b = P[2:, 1:-1] - P[:-2, 1:-1]
    na, nb = np.linalg.norm(a, axis=-1), np.linalg.norm(b, axis=-1)
    sin = np.linalg.norm(np.cross(b, a), axis=-1) / np.maximum(na * nb, 1e-300)
    r = np.sqrt(rx ** 2 + ry ** 2)[1:-1, 1:-1]
    dd = rel * np.abs(depth[1:-1, 1:-1]) * (1 + r)
    with np.errstate(divide="ignore", invalid="ignore"):
        kap[1:-1, 1:-1] = (dd / na + dd / nb) / sin
    return np.nan_to_num(kap, nan=np.inf)


def _dist_tol(ref):
    w, d = ref["weights"], ref["d_all"]
    W = w.sum(1)
    m = (w * d).sum(1) / np.maximum(W, 1e-30)
    dmax = np.where(w > 0, np.abs(d), 0).max(1, initial=0)
    spread = (w * np.abs(d - m[:, None])).sum(1)
    return 1e-4 * np.abs(ref["dist"]) + 1e-4 * W * spread * dmax + 1e-7 * W * W * dmax ** 2


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 8)])
def test_loss_maps_match_oracle(tile):
    sc, cam = scenes.tiny_scene(), _cam()
    p = RenderParams(tile_w=tile[0], tile_h=tile[1], losses=True)
    fr = _frame(sc, cam, p)
    ref, _, _ = olosses.render_with_losses(sc, cam, None, oracle_params(p))
    H, W = cam.height, cam.width
    pix = np.arange(H * W)
    # the four standard maps are unchanged by the loss state
    bad, rep = compare_maps(gpu_maps_at(fr, pix), ref, ref["margin"])
    assert rep["n_bad"] == 0 and rep["ambiguous"] < 1e-2, rep
    dist, nloss = [t.cpu().numpy().reshape(-1) for t in fr.loss_maps(0)]
    amb = (ref["margin"] < AMBIG_MARGIN).reshape(H, W)
    ok = ~amb.reshape(-1)
    err = np.abs(dist - ref["dist"])
    assert (err[ok] <= _dist_tol(ref)[ok]).all(), float((err / np.maximum(_dist_tol(ref), 1e-30))[ok].max())
    assert (ref["dist"] > 1e-3).sum() > 500      # the map is not trivially zero
    # normal consistency: pixels whose stencil is unambiguous and well conditioned
    kap = _conditioning(ref["depth"].reshape(H, W), cam).reshape(-1)
    sel = ~_dilate(amb).reshape(-1) & ((kap < 1e-2) | ~ref["n_ok"])
    assert sel.mean() > 0.8 and (ref["n_ok"] & sel).sum() > 3000
    N = np.linalg.norm(ref["normal"], axis=1)
    tol = 1e-4 + 4 * N * np.where(ref["n_ok"], kap, 0)
    en = np.abs(nloss - ref["nloss"])
    assert (en[sel] <= tol[sel]).all(), (float(en[sel].max()), int((en[sel] > tol[sel]).sum()))


def test_normal_consistency_stencil_on_the_gpu_maps():
    # the same GPU depth / alpha / normal maps through the oracle's Eq. 24
    sc, cam = scenes.tiny_scene(seed=4), _cam()
    p = RenderParams(losses=True)
    fr = _frame(sc, cam, p)
    c, a, d, n = [t.cpu().numpy().astype(np.float64) for t in fr.view_maps(0)]
    nt, okm = olosses.depth_normals(torch.from_numpy(d), torch.from_numpy(a), cam)
    nt = nt.numpy()
    ref = np.where(okm.numpy(), a - (n.transpose(1, 2, 0) * nt).sum(-1), 0.0)
    got = fr.loss_maps(0)[1].cpu().numpy()
    kap = _conditioning(d, cam, rel=1e-7)    # FP32 rounding of the stencil itself
    sel = kap < 1e-2
    assert okm.numpy().sum() > 3000
    np.testing.assert_array_less(np.abs(got - ref)[sel], 1e-4 + 8 * np.linalg.norm(n, axis=0)[sel] * kap[sel])
    assert (got[~okm.numpy()] == 0).all()


@pytest.mark.parametrize("which", ["dist", "nloss", "all"])
def test_loss_gradients_match_oracle(which):
    sc, cam = scenes.tiny_scene(seed=2), _cam()
    H, W = cam.height, cam.width
    p = RenderParams(losses=True)
    op = oracle_params(p)
    ref0, _, _ = olosses.render_with_losses(sc, cam, None, op)
    amb = (ref0["margin"] < AMBIG_MARGIN).reshape(H, W)
    kap = _conditioning(ref0["depth"].reshape(H, W), cam)
    ln_bad = _dilate(amb) | (ref0["n_ok"].reshape(H, W) & (kap > 1e-3))
    base = [u[0] for u in scenes.upstream_grads(11, H, W)]
    ld, ln = [u[0] for u in scenes.loss_upstream(12, H, W)]
    zero = lambda u: np.zeros_like(u)
    if which != "all":
        base = [zero(u) for u in base]
    if which == "dist":
        ln = zero(ln)
    if which == "nloss":
        ld = zero(ld)
    mask2 = lambda u, m: np.where(m, 0.0, u).astype(np.float32)
    up = [mask2(base[0], amb[None]), mask2(base[1], amb), mask2(base[2], amb), mask2(base[3], amb[None]),
          mask2(ld, amb), mask2(ln, ln_bad)]
    pg, g2, sp, s2 = oracle_grads_with_spread(sc, cam, up, op,
                                              fn=lambda s: olosses.render_with_losses(s, cam, up, op)[1:])
    fr = _frame(sc, cam, p)
    t = [torch.from_numpy(u).to(DEV) for u in up]
    grads = fr.backward(*t[:4], ddist=t[4], dnloss=t[5])[0]
    torch.cuda.synchronize()
    dbg = fr.debug()["grad2d"].cpu().numpy()
    r0 = oracle.render(sc, cam, op, pixels=np.array([0]))
    v = r0["dec"]["valid"]   # culled entries' rows of the 2D-gradient buffer are never written
    rec = grad2d_to_record(dbg[v], {k: r0["pre"][k][v] for k in ("conic", "p", "opacity")})
    g2_gpu = {k: rec[k].reshape(g2[k][v].shape) for k in rec}
    g2 = {k: g2[k][v] for k in g2}
    s2 = {k: s2[k][v] for k in s2}
    const = ("conic", "opacity", "rgb", "n") if which == "dist" else ()
    for k in const:   # Eq. 23's weights are constants: nothing reaches them
        assert np.abs(g2_gpu[k]).max() == 0 and np.abs(g2[k]).max() == 0, k
    assert_grads_close({k: g2_gpu[k] for k in rec if k not in const}, {k: g2[k] for k in rec if k not in const},
                       s2, what="2D gradients")
    skip = ("opacities", "sh") if which == "dist" else ()
    assert_grads_close({k: g.cpu().numpy() for k, g in grads.items() if k not in skip},
                       {k: v for k, v in pg.items() if k not in skip}, sp, what="parameter gradients")


def test_loss_state_leaves_the_plain_gradients_unchanged():
    # losses on, ddist = dnloss = NULL: the same kernels as without the loss state
    sc, cam = scenes.tiny_scene(seed=3), _cam()
    up = [torch.from_numpy(u[0]).to(DEV) for u in scenes.upstream_grads(5, cam.height, cam.width)]
    outs = []
    for losses in (False, True):
        fr = _frame(sc, cam, RenderParams(losses=losses))
        g = fr.backward(*up)[0]
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in g.items()})
    for k in outs[0]:
        s = np.abs(outs[0][k]).max()
        np.testing.assert_allclose(outs[1][k], outs[0][k], rtol=0, atol=1e-5 * s)


def test_multi_view_loss_maps_match_single_views():
    sc = scenes.tiny_scene(seed=5)
    cams = [_cam(), scenes.tiny_camera()]
    p = RenderParams(losses=True)
    st = SceneTensors.from_scene(sc, DEV)
    fr = Frame([st], [(c, 0) for c in cams], p)
    fr.forward()
    singles = [_frame(sc, c, p) for c in cams]
    for v, s in enumerate(singles):
        for a, b in zip(fr.loss_maps(v), s.loss_maps(0)):
            torch.testing.assert_close(a, b, rtol=0, atol=0)
