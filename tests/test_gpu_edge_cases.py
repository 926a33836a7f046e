"""More parity cases of the CUDA path against the FP64 oracle: every SH degree
(the kernels are instantiated per degree), BF16 rows that are not a multiple
of 16 bytes, a splat whose rectangle covers the whole image, and the bounded
device waits' timeout status."""
import numpy as np
import pytest
import torch

import oracle
from oracle import binning
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, _lib, scenes
from tests._util import assert_grads_close, oracle_grads_with_spread, _same_ranges, AMBIG_MARGIN, compare_maps, gpu_maps_at, oracle_params

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _with_degree(sc, deg, seed):
    """The scene with SH of degree deg: its DC term kept, higher bands N(0, 0.2)."""
    rng = np.random.default_rng(seed)
    K = (deg + 1) ** 2
    sh = np.zeros((sc.n, K, 3), np.float32)
    sh[:, 0] = sc.sh[:, 0]
    sh[:, 1:] = rng.normal(0.0, 0.2, (sc.n, K - 1, 3))
    return scenes.Scene(sc.means, sc.scales, sc.quats, sc.opacities, sh, deg)


def _small_camera():
    # ragged for 16x16 tiles, off-centre principal point
    return scenes.Camera(scenes.look_at((0.4, -0.3, -0.6), (0.0, 0.0, 3.0)), 90.0, 90.0, 41.0, 29.5, 83, 61)


def _frame(sc, cam, p, dtype=torch.float32):
    fr = Frame([SceneTensors.from_scene(sc, DEV, dtype)], [(cam, 0)], p)
    fr.forward()
    torch.cuda.synchronize()
    return fr


def _check_all(sc, cam, p, fr, seed):
    op = oracle_params(p)
    dec = binning.decide_scene(sc, cam, op)
    tile_ref, g_ref, ranges_ref = binning.tile_lists(dec, cam, op)
    dbg = fr.debug()
    np.testing.assert_array_equal(dbg["pair_tile"].cpu().numpy(), tile_ref)
    np.testing.assert_array_equal(dbg["pair_entry"].cpu().numpy(), g_ref)
    _same_ranges(dbg["ranges"].cpu().numpy(), ranges_ref)
    ref = oracle.render(sc, cam, op)
    bad, rep = compare_maps(gpu_maps_at(fr, np.arange(cam.width * cam.height)), ref, ref["margin"])
    assert rep["n_bad"] == 0 and rep["ambiguous"] < 1e-2, rep
    amb = (ref["margin"] < AMBIG_MARGIN).reshape(cam.height, cam.width)
    up = [u[0] for u in scenes.upstream_grads(seed, cam.height, cam.width)]
    up = [np.where(amb if u.ndim == 2 else amb[None], 0.0, u).astype(np.float32) for u in up]
    pg, _, sp, _ = oracle_grads_with_spread(sc, cam, up, op)
    g = fr.backward(*[torch.from_numpy(u).to(DEV) for u in up])[0]
    torch.cuda.synchronize()
    for k in pg:
        assert np.abs(pg[k]).max() > 0, k
    assert_grads_close({k: v.cpu().numpy() for k, v in g.items()}, pg, sp, what="parameter gradients")
    return dbg, g


@pytest.mark.parametrize("deg", [0, 1, 2, 3])
def test_every_sh_degree_matches_oracle(deg):
    sc = _with_degree(scenes.tiny_scene(900, seed=11), deg, seed=deg)
    cam = _small_camera()
    p = RenderParams()
    _check_all(sc, cam, p, _frame(sc, cam, p), seed=30 + deg)


@pytest.mark.parametrize("deg", [0, 3])
def test_clamped_colour_channels_match_oracle(deg):
    """A third of the splats have their red channel below 0 before the clamp
    rgb = max(SH + 1/2, 0): the forward records red 0 for them, no gradient
    reaches their red SH coefficients where the clamp holds, and every map and
    gradient matches the oracle (which differentiates through the clamp)."""
    sc = _with_degree(scenes.tiny_scene(900, seed=12), deg, seed=40 + deg)
    sh = sc.sh.copy()
    third = np.arange(sc.n) % 3 == 0
    sh[third, 0, 0] = (-0.3 - 0.5) / scenes.Y00   # red -0.3 before the clamp (degree 0)
    sc = scenes.Scene(sc.means, sc.scales, sc.quats, sc.opacities, sh, deg)
    cam = _small_camera()
    p = RenderParams()
    dbg, g = _check_all(sc, cam, p, _frame(sc, cam, p), seed=50 + deg)
    rec = dbg["rec"].cpu().numpy()
    vis = np.zeros(sc.n, bool)
    vis[np.unique(dbg["pair_entry"].cpu().numpy())] = True
    red_clamped = vis & (rec[:, 12] == 0.0)
    assert red_clamped.sum() >= 20, red_clamped.sum()   # the clamp engages on visible splats
    if deg == 0:   # no higher band can lift red above 0: exactly the chosen third
        assert np.array_equal(red_clamped, vis & third)
        assert np.all(g["sh"].cpu().numpy()[vis & third, 0, 0] == 0.0)


@pytest.mark.parametrize("deg", [1, 2])
def test_bf16_rows_of_any_length_match_fp32_on_rounded_inputs(deg):
    # BF16 SH rows are 24 B (degree 1) and 54 B (degree 2): neither is a whole
    # number of 16-byte pieces, so the loads take the element-wise path
    sc = _with_degree(scenes.tiny_scene(900, seed=12), deg, seed=10 + deg)
    r = scenes.to_bf16_rounded
    sc_r = scenes.Scene(r(sc.means), r(sc.scales), r(sc.quats), r(sc.opacities), r(sc.sh), deg)
    cam = _small_camera()
    p = RenderParams()
    a = _frame(sc, cam, p, torch.bfloat16)
    b = _frame(sc_r, cam, p)
    for x, y in zip(a.view_maps(0), b.view_maps(0)):
        torch.testing.assert_close(x, y, rtol=0, atol=0)
    up = [torch.from_numpy(u[0]).to(DEV) for u in scenes.upstream_grads(40 + deg, cam.height, cam.width)]
    ga, gb = a.backward(*up)[0], b.backward(*up)[0]
    torch.cuda.synchronize()
    for k in gb:   # same FP32 arithmetic after widening; float atomics may add in another order
        torch.testing.assert_close(ga[k], gb[k], rtol=1e-4, atol=1e-5 * gb[k].abs().max().item())


def test_splat_covering_the_whole_image():
    # one wide splat close to the camera touches every tile; small ones in front
    # of and behind it
    sc = _with_degree(scenes.tiny_scene(300, seed=13), 1, seed=5)
    big = scenes.Scene(np.array([[0.05, -0.02, 1.5]], np.float32), np.array([[1.2, 0.9, 0.4]], np.float32),
                       np.array([[0.9, 0.2, -0.1, 0.3]], np.float32), np.array([0.6], np.float32),
                       np.full((1, 4, 3), 0.1, np.float32), 1)
    cat = lambda f: np.concatenate([getattr(sc, f), getattr(big, f)])
    sc = scenes.Scene(cat("means"), cat("scales"), cat("quats"), cat("opacities"), cat("sh"), 1)
    sc.means[:150, 2] *= 0.5   # half of the small ones in front of it (z in [1, 2])
    cam = _small_camera()
    for tile in [(16, 16), (8, 8)]:
        p = RenderParams(tile_w=tile[0], tile_h=tile[1])
        fr = _frame(sc, cam, p)
        dec = binning.decide_scene(sc, cam, oracle_params(p))
        r = dec["rect"][-1]
        assert dec["valid"][-1] and r[0] == 0 and r[1] == cam.width - 1 and r[2] == 0 and r[3] == cam.height - 1
        _check_all(sc, cam, p, fr, seed=50)


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    # a device wait on a word that nothing publishes gives up after its poll
    # limit, sets GS_ERR_TIMEOUT and returns: no hang, no fault
    sc, cam = scenes.tiny_scene(500, seed=14), scenes.tiny_camera()
    p = RenderParams()
    fr = _frame(sc, cam, p)
    before = [t.clone() for t in fr.view_maps(0)]
    assert fr.stats().status == 0
    fr.debug_wait_timeout(1000)
    torch.cuda.synchronize()
    assert fr.stats().status == _lib.GS_ERR_TIMEOUT
    fr.forward()   # the next frame clears the status and renders as before
    torch.cuda.synchronize()
    assert fr.stats().status == 0
    for a, b in zip(before, fr.view_maps(0)):
        torch.testing.assert_close(a, b, rtol=0, atol=0)
