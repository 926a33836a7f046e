"""Decoupled appearance on the GPU (gs_appearance_fwd_bwd, gs_adam_step) against
the FP64 oracle, and its training on rendered views with per-view exposure and
white-balance shifts."""
import numpy as np
import pytest
import torch

from tests._util import assert_grads_close

from oracle import appearance as oapp
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes
from paper_2406_01467_b300.appearance import Appearance, adam_step

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _frame(n_views=3):
    sc = scenes.object_scene(30_000, seed=41)
    cams = scenes.fusion_cameras(n_views, seed=5, radius=4.0, width=173, height=131)
    fr = Frame([SceneTensors.from_scene(sc, DEV)], [(c, 0) for c in cams], RenderParams())
    fr.forward()
    torch.cuda.synchronize()
    return fr, cams


def _split(flat, cams):
    out, off = [], 0
    for c in cams:
        n = 3 * c.width * c.height
        out.append(flat[off:off + n].reshape(3, c.height, c.width))
        off += n
    return out


def _targets(colors, seed):
    rng = np.random.default_rng(seed)
    out = []
    for c in colors:
        g = rng.uniform(0.7, 1.3, 3)
        o = rng.uniform(-0.05, 0.05, 3)
        out.append((g[:, None, None] * c + o[:, None, None]).astype(np.float32))
    return out


def test_one_call_matches_oracle():
    fr, cams = _frame(3)
    app = Appearance(5, embed_dim=16, hidden=32, seed=1)
    rng = np.random.default_rng(0)
    app.params.copy_(torch.from_numpy(rng.normal(0, 0.3, app.params.numel()).astype(np.float32)))
    col = fr.color.clone()
    cols = _split(col.cpu().numpy(), cams)
    tg = _targets(cols, 1)
    target = torch.from_numpy(np.concatenate([t.ravel() for t in tg])).to(DEV)
    corrected = torch.empty_like(col)
    idx = [4, 0, 2]
    loss, dcol = app.fwd_bwd(fr, idx, col, target, corrected)
    torch.cuda.synchronize()
    l_ref, g_ref, dc_ref, corr_ref = oapp.loss_and_grads(app.params.cpu().numpy(), 5, 16, 32, cols, tg, idx)
    np.testing.assert_allclose(loss.cpu().numpy(), l_ref, rtol=1e-5)
    for a, b in zip(_split(corrected.cpu().numpy(), cams), corr_ref):
        np.testing.assert_allclose(a, b, atol=2e-6)
    # dL/dc: exact sign decisions except where |c' - target| is at rounding level
    mask = [np.abs(c - t) > 1e-5 for c, t in zip(corr_ref, tg)]
    for a, b, m in zip(_split(dcol.cpu().numpy(), cams), dc_ref, mask):
        ok = m.all(axis=0)[None].repeat(3, 0)
        # terms of size 1/(3HW) cancel: absolute tolerance on that scale
        np.testing.assert_allclose(a[ok], b[ok], rtol=1e-5, atol=1e-5 * np.abs(b).max())
    assert_grads_close({"params": app.grads.cpu().numpy()}, {"params": g_ref}, what="appearance gradients")


def test_adam_matches_oracle():
    rng = np.random.default_rng(3)
    n = 10_000
    p = rng.normal(size=n).astype(np.float32)
    P, M, V = torch.from_numpy(p).to(DEV), torch.zeros(n, device=DEV), torch.zeros(n, device=DEV)
    pr, mr, vr = p.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 6):
        g = rng.normal(size=n).astype(np.float32)
        G = torch.from_numpy(g).to(DEV)
        adam_step(P, G, M, V, step, lr=1e-2)
        pr, mr, vr = oapp.adam(pr, g.astype(np.float64), mr, vr, step, lr=1e-2)
        assert torch.count_nonzero(G) == 0
    np.testing.assert_allclose(P.cpu().numpy(), pr, rtol=1e-5, atol=1e-6)


def test_training_removes_exposure_and_white_balance():
    fr, cams = _frame(4)
    col = fr.color.clone()
    cols = _split(col.cpu().numpy(), cams)
    tg = _targets(cols, 2)
    target = torch.from_numpy(np.concatenate([t.ravel() for t in tg])).to(DEV)
    app = Appearance(4, embed_dim=16, hidden=32, seed=3)
    corrected = torch.empty_like(col)
    before = np.mean([oapp.psnr(c, t) for c, t in zip(cols, tg)])
    for it in range(300):
        loss, dcol = app.fwd_bwd(fr, range(4), col, target, corrected)
        app.step(lr=1e-2)
    torch.cuda.synchronize()
    after = np.mean([oapp.psnr(c, t) for c, t in zip(_split(corrected.cpu().numpy(), cams), tg)])
    print(f"appearance PSNR {before:.2f} -> {after:.2f} dB")
    assert after > before + 10, (before, after)
    # the corrected-colour gradient drives the rasterizer backward (joint step)
    g = fr.backward(dcol)[0]
    torch.cuda.synchronize()
    assert all(torch.isfinite(t).all() for t in g.values()) and g["sh"].abs().max() > 0
