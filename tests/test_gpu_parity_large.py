"""Parity at the workload sizes (object scene 200K / 800x600, unbounded scene
3M / 1297x840 in the launch configuration the benchmark times), and the edge
cases: empty and culled scenes, ragged images, non-finite inputs, capacity
overflow, BF16 storage, several views of several scenes in one frame."""
import numpy as np
import pytest
import torch

import oracle
from oracle import binning
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes
from paper_2406_01467_b300 import _lib
from tests._util import (_same_ranges, AMBIG_MARGIN, assert_grads_close, compare_maps, gpu_maps_at,
                         oracle_grads_with_spread, oracle_params)

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _frame(scene, cam, params, cap=None, dtype=torch.float32):
    fr = Frame([SceneTensors.from_scene(scene, DEV, dtype)], [(cam, 0)], params, cap)
    fr.forward()
    torch.cuda.synchronize()
    return fr


def _crops(cam, n, size, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        x0 = int(rng.integers(0, cam.width - size))
        y0 = int(rng.integers(0, cam.height - size))
        ys, xs = np.mgrid[y0:y0 + size, x0:x0 + size]
        out.append((ys * cam.width + xs).reshape(-1))
    return out


def _check_tile_lists(fr, scene, cam, p):
    op = oracle_params(p)
    dec = binning.decide(scene.means, scene.scales, scene.quats, scene.opacities, cam, op)
    tile_ref, g_ref, ranges_ref = binning.tile_lists(dec, cam, op)
    dbg = fr.debug()
    assert dbg["stats"].n_pairs == len(tile_ref)
    assert dbg["stats"].n_visible == int(dec["valid"].sum())
    np.testing.assert_array_equal(dbg["pair_tile"].cpu().numpy(), tile_ref)
    np.testing.assert_array_equal(dbg["pair_entry"].cpu().numpy(), g_ref)
    _same_ranges(dbg["ranges"].cpu().numpy(), ranges_ref)
    return dec


def _reaching(dec, cam, pix):
    """Indices of the valid Gaussians whose pixel rectangle meets the crop's box.
    Per-pixel results depend on these only (decisions are per Gaussian, and a
    subset keeps the index order that breaks depth ties)."""
    x0, x1 = pix.min() % cam.width, pix.max() % cam.width
    y0, y1 = pix.min() // cam.width, pix.max() // cam.width
    r = dec["rect"]
    return np.nonzero(dec["valid"] & (r[:, 1] >= x0) & (r[:, 0] <= x1) & (r[:, 3] >= y0) & (r[:, 2] <= y1))[0]


def _check_crops(fr, scene, cam, p, crops, max_ambig=0.02, dec=None):
    op = oracle_params(p)
    for pix in crops:
        sub = scene if dec is None else scene.subset(_reaching(dec, cam, pix))
        ref = oracle.render(sub, cam, op, pixels=pix)
        bad, rep = compare_maps(gpu_maps_at(fr, pix), ref, ref["margin"])
        assert rep["ambiguous"] <= max_ambig, rep
        assert rep["n_bad"] == 0, rep


def _grads_on_crop(fr, scene, cam, p, pix, dec, seed=3):
    """GPU gradients with the upstream gradient restricted to one crop, against
    the oracle over the Gaussians that can reach the crop, entry by entry."""
    op = oracle_params(p)
    up = [u[0] for u in scenes.upstream_grads(seed, cam.height, cam.width)]
    sel = _reaching(dec, cam, pix)
    sub = scene.subset(sel)
    ref_f = oracle.render(sub, cam, op, pixels=pix)
    keep = np.zeros(cam.width * cam.height, bool)
    keep[pix[ref_f["margin"] >= AMBIG_MARGIN]] = True
    m = keep.reshape(cam.height, cam.width)
    up = [(u * (m if u.ndim == 2 else m[None])).astype(np.float32) for u in up]
    grads = fr.backward(*[torch.from_numpy(u).to(DEV) for u in up])[0]
    torch.cuda.synchronize()
    pg, _, sp, _ = oracle_grads_with_spread(sub, cam, up, op, pixels=pix)
    gpu, ref, spread = {}, {}, {}
    for k in ("means", "scales", "quats", "opacities", "sh"):
        g = grads[k].cpu().numpy()
        r = np.zeros_like(g, dtype=np.float64)
        e = np.zeros_like(g, dtype=np.float64)
        r[sel], e[sel] = pg[k], sp[k]
        assert np.abs(r).max() > 0, k
        gpu[k], ref[k], spread[k] = g, r, e
    # every other Gaussian gets exactly zero
    return assert_grads_close(gpu, ref, spread, what=f"crop at pixel {int(pix[0])}")


def _clamp_crops(scene, cam, p, dec, size=16):
    """Crops on the image border where splats whose J is clamped (centre beyond
    the image widened by clamp_margin) contribute: top, left and bottom edges and
    the bottom-right corner of the 1297x840 view."""
    from oracle.params import clamp_limits_f32
    lims = clamp_limits_f32(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, p.clamp_margin)
    tx = (dec["u"].astype(np.float64) - cam.cx) / cam.fx
    ty = (dec["v"].astype(np.float64) - cam.cy) / cam.fy
    clamped = dec["valid"] & ((tx < lims[0]) | (tx > lims[1]) | (ty < lims[2]) | (ty > lims[3]))
    W, H = cam.width, cam.height
    out = []
    for x0, y0 in ((560, 0), (0, 100), (400, H - size), (W - size - 5, H - size - 4)):
        ys, xs = np.mgrid[y0:y0 + size, x0:x0 + size]
        pix = (ys * W + xs).reshape(-1)
        hit = np.intersect1d(_reaching(dec, cam, pix), np.nonzero(clamped)[0])
        assert len(hit) > 0, (x0, y0)
        out.append(pix)
    return out


def test_object_scale_parity():
    sc, cam = scenes.object_scene(), scenes.object_camera()
    p = RenderParams()
    fr = _frame(sc, cam, p)
    dec = _check_tile_lists(fr, sc, cam, p)
    crops = _crops(cam, 4, 24, seed=5)
    _check_crops(fr, sc, cam, p, crops, dec=dec)
    for i, pix in enumerate(crops[:2]):
        _grads_on_crop(fr, sc, cam, p, pix, dec, seed=3 + i)


@pytest.mark.slow
def test_unbounded_parity_bench_configuration():
    sc, cam = scenes.unbounded_scene(), scenes.unbounded_camera()
    p = RenderParams()   # the benchmark's configuration: 16x16 tiles, defaults
    fr = _frame(sc, cam, p)
    dec = _check_tile_lists(fr, sc, cam, p)
    crops = _crops(cam, 3, 16, seed=9)
    border = _clamp_crops(sc, cam, p, dec)
    _check_crops(fr, sc, cam, p, crops + border, max_ambig=0.05, dec=dec)
    for i, pix in enumerate(crops[:1] + border):
        _grads_on_crop(fr, sc, cam, p, pix, dec, seed=3 + i)


def test_empty_scene():
    sc = scenes.tiny_scene(0)
    cam = scenes.tiny_camera()
    fr = _frame(sc, cam, RenderParams())
    for t in fr.view_maps(0):
        assert torch.count_nonzero(t).item() == 0
    g = fr.backward(torch.ones(3, 128, 128, device=DEV))[0]
    assert g["means"].numel() == 0
    assert fr.stats().status == 0


def test_all_culled():
    sc = scenes.tiny_scene(500)
    sc.means[:, 2] = -3.0    # behind the camera
    fr = _frame(sc, scenes.tiny_camera(), RenderParams())
    st = fr.stats()
    assert st.n_visible == 0 and st.n_pairs == 0 and st.status == 0
    assert torch.count_nonzero(fr.view_maps(0)[1]).item() == 0
    g = fr.backward(torch.ones(3, 128, 128, device=DEV), torch.ones(128, 128, device=DEV))[0]
    assert torch.count_nonzero(g["means"]).item() == 0


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (32, 4)])
def test_ragged_image(tile):
    sc = scenes.tiny_scene(800, seed=4)
    cam = scenes.Camera(np.eye(4), 40.0, 40.0, 18.5, 11.0, 37, 23)
    p = RenderParams(tile_w=tile[0], tile_h=tile[1])
    fr = _frame(sc, cam, p)
    _check_tile_lists(fr, sc, cam, p)
    ref = oracle.render(sc, cam, oracle_params(p))
    bad, rep = compare_maps(gpu_maps_at(fr, np.arange(37 * 23)), ref, ref["margin"])
    assert rep["n_bad"] == 0, rep


def test_single_gaussian_peak_alpha_is_opacity_on_gpu():
    # P1 through the CUDA path: centre on a pixel centre -> alpha = o, colour = o rgb.
    cam = scenes.Camera(np.eye(4), 64.0, 64.0, 16.0, 16.0, 32, 32)
    z = 2.0
    m = np.array([[(10.5 - 16) * z / 64.0, (20.5 - 16) * z / 64.0, z]], np.float32)
    sc = scenes.Scene(m, np.array([[0.05, 0.03, 0.02]], np.float32), np.array([[0.9, 0.1, -0.2, 0.3]], np.float32),
                      np.array([0.7], np.float32), np.zeros((1, 1, 3), np.float32), 0)
    fr = _frame(sc, cam, RenderParams())
    c, a, d, n = [t.cpu().numpy() for t in fr.view_maps(0)]
    assert abs(a[20, 10] - np.float32(0.7)) < 1e-6
    np.testing.assert_allclose(c[:, 20, 10], 0.7 * 0.5, atol=1e-6)
    assert abs(d[20, 10] - z) < 1e-6


def test_nonfinite_inputs_are_culled_and_reported():
    sc = scenes.tiny_scene(300, seed=2)
    bad = sc.subset(np.arange(300))
    bad.means[7, 0] = np.nan
    bad.scales[11, 1] = np.inf
    bad.sh[13, 0, 2] = np.nan
    cam = scenes.tiny_camera()
    st = SceneTensors.from_scene(bad, DEV)
    fr = Frame([st], [(cam, 0)], RenderParams())
    fr.forward()
    s = fr.stats()
    assert fr.last_status == _lib.GS_ERR_NUMERIC and s.n_nonfinite == 3
    keep = np.setdiff1d(np.arange(300), [7, 11, 13])
    good = _frame(sc.subset(keep), cam, RenderParams())
    for a, b in zip(fr.view_maps(0), good.view_maps(0)):
        torch.testing.assert_close(a, b, rtol=0, atol=0)


def test_capacity_overflow_is_detected_then_grown():
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams()
    fr = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p, pair_capacity=100)
    fr.preprocess()
    fr.bin()
    fr.render()
    s = fr.stats()
    assert fr.last_status == _lib.GS_ERR_CAPACITY and s.n_pairs > 100
    fr.forward()   # grows the workspace and renders again
    assert fr.stats().status == 0
    ref = _frame(sc, cam, p)
    for a, b in zip(fr.view_maps(0), ref.view_maps(0)):
        torch.testing.assert_close(a, b, rtol=0, atol=0)


def test_bf16_storage_matches_oracle_on_rounded_params():
    sc = scenes.object_scene(20_000, seed=3)
    cam = scenes.object_camera(320, 240, 440.0)
    r = lambda a: scenes.to_bf16_rounded(a)
    sc_r = scenes.Scene(r(sc.means), r(sc.scales), r(sc.quats), r(sc.opacities), r(sc.sh), sc.sh_degree)
    p = RenderParams()
    fr = _frame(sc, cam, p, dtype=torch.bfloat16)
    ref_fr = _frame(sc_r, cam, p)
    for a, b in zip(fr.view_maps(0), ref_fr.view_maps(0)):   # same FP32 arithmetic after widening
        torch.testing.assert_close(a, b, rtol=0, atol=0)
    _check_crops(fr, sc_r, cam, p, _crops(cam, 2, 24, seed=1))


def test_several_views_and_scenes_in_one_frame():
    a, b = scenes.tiny_scene(1500, seed=5), scenes.object_scene(8000, seed=6)
    cam_a = scenes.tiny_camera()
    cam_b = scenes.object_camera(200, 150, 275.0)
    cam_a2 = scenes.Camera(scenes.look_at((0.3, 0.0, -0.5), (0.0, 0.0, 3.0)), 100.0, 100.0, 48.0, 40.0, 96, 80)
    p = RenderParams()
    sa, sb = SceneTensors.from_scene(a, DEV), SceneTensors.from_scene(b, DEV)
    fr = Frame([sa, sb], [(cam_a, 0), (cam_b, 1), (cam_a2, 0)], p)
    fr.forward()
    singles = [_frame(a, cam_a, p), _frame(b, cam_b, p), _frame(a, cam_a2, p)]
    for v, s in enumerate(singles):
        for x, y in zip(fr.view_maps(v), s.view_maps(0)):
            torch.testing.assert_close(x, y, rtol=0, atol=0)
    # gradients: a scene seen by two views gets the sum of both views' gradients
    ups = []
    for v, (h, w) in enumerate(fr.sizes):
        u = scenes.upstream_grads(20 + v, h, w)
        ups.append([torch.from_numpy(x[0]).to(DEV) for x in u])
    cat = [torch.cat([u[k].reshape(-1) for u in ups]) for k in range(4)]
    g = fr.backward(*cat)
    gs = [s.backward(*u)[0] for s, u in zip(singles, ups)]
    torch.cuda.synchronize()
    for k in g[0]:
        ref_a = gs[0][k] + gs[2][k]
        torch.testing.assert_close(g[0][k], ref_a, rtol=1e-4, atol=1e-5 * ref_a.abs().max().item())
        # float atomics add in a different order: equal up to rounding
        torch.testing.assert_close(g[1][k], gs[1][k], rtol=1e-4, atol=1e-5 * gs[1][k].abs().max().item())


def test_forward_is_deterministic():
    sc, cam = scenes.object_scene(50_000, seed=8), scenes.object_camera(400, 300, 550.0)
    p = RenderParams()
    a = _frame(sc, cam, p)
    b = _frame(sc, cam, p)
    for x, y in zip(a.view_maps(0), b.view_maps(0)):
        torch.testing.assert_close(x, y, rtol=0, atol=0)
