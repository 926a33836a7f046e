"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tile lists and sort order: bit-exact.  Colour, alpha, normal: 1e-4 absolute;
depth: 1e-4 relative, on pixels whose discrete decisions are not within the
FP32/FP64 ambiguity margin.  Gradients: every entry within 1e-3 relative plus
16 times the change FP32 evaluations of the oracle make to it (tests/_util.py).
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import binning
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes
from tests._util import (_same_ranges, AMBIG_MARGIN, assert_grads_close, compare_maps, gpu_maps_at,
                         grad2d_to_record, oracle_grads_with_spread, oracle_params)

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _frame(scene, cam, params, cap=None):
    st = SceneTensors.from_scene(scene, DEV)
    fr = Frame([st], [(cam, 0)], params, cap)
    fr.forward()
    torch.cuda.synchronize()
    return fr


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 8), (32, 8)])
def test_tile_lists_bit_exact_tiny(tile):
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams(tile_w=tile[0], tile_h=tile[1])
    fr = _frame(sc, cam, p)
    dbg = fr.debug()
    op = oracle_params(p)
    dec = binning.decide(sc.means, sc.scales, sc.quats, sc.opacities, cam, op)
    tile_ref, g_ref, ranges_ref = binning.tile_lists(dec, cam, op)
    rect = dbg["rect"].cpu().numpy()
    valid = rect[:, 1] >= rect[:, 0]
    np.testing.assert_array_equal(valid, dec["valid"])
    np.testing.assert_array_equal(rect[valid], dec["rect"][valid])
    np.testing.assert_array_equal(dbg["pair_tile"].cpu().numpy(), tile_ref)
    np.testing.assert_array_equal(dbg["pair_entry"].cpu().numpy(), g_ref)
    _same_ranges(dbg["ranges"].cpu().numpy(), ranges_ref)
    assert dbg["stats"].n_pairs == len(tile_ref)


def test_records_match_oracle_tiny():
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams()
    fr = _frame(sc, cam, p)
    rec = fr.debug()["rec"].cpu().numpy()
    ref = oracle.render(sc, cam, oracle_params(p), pixels=np.array([0]))
    v = ref["dec"]["valid"]
    pre = ref["pre"]
    np.testing.assert_allclose(rec[v, 0], pre["u"][v], atol=1e-4)
    np.testing.assert_allclose(rec[v, 1], pre["v"][v], atol=1e-4)
    # the record's conic is scaled for base-2 exponentials: log2(e) (a / 2, b, c / 2)
    kscale = np.log2(np.e) * np.array([0.5, 1.0, 0.5])
    for k, col in enumerate((2, 3, 4)):
        scale = np.abs(pre["conic"][v]).max(axis=1) * kscale[k]
        np.testing.assert_array_less(np.abs(rec[v, col] - kscale[k] * pre["conic"][v, k]), 1e-4 * scale + 1e-9)
    np.testing.assert_allclose(rec[v, 5], pre["opacity"][v], rtol=1e-7)
    np.testing.assert_allclose(rec[v, 10], pre["z"][v], rtol=1e-6)
    np.testing.assert_allclose(rec[v, 8:10], pre["p"][v], atol=1e-5)
    np.testing.assert_allclose(rec[v][:, [15, 6, 7]], pre["n"][v], atol=1e-5)   # (n_x | n_y, n_z)
    np.testing.assert_allclose(rec[v, 12:15], pre["rgb"][v], atol=1e-5)
    assert (rec[v, 11] == 0).all()


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 8)])
def test_forward_maps_tiny(tile):
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams(tile_w=tile[0], tile_h=tile[1])
    fr = _frame(sc, cam, p)
    pixels = np.arange(cam.width * cam.height)
    ref = oracle.render(sc, cam, oracle_params(p))
    bad, rep = compare_maps(gpu_maps_at(fr, pixels), ref, ref["margin"])
    assert rep["ambiguous"] < 1e-2, rep
    assert rep["n_bad"] == 0, rep


def test_forward_is_tile_size_independent():
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    outs = []
    for tile in [(16, 16), (8, 8), (32, 8)]:
        fr = _frame(sc, cam, RenderParams(tile_w=tile[0], tile_h=tile[1]))
        outs.append([t.cpu().numpy() for t in fr.view_maps(0)])
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            np.testing.assert_array_equal(a, b)


def _upstream(cam, seed, ambiguous_mask=None):
    up = [u[0] for u in scenes.upstream_grads(seed, cam.height, cam.width)]
    if ambiguous_mask is not None:
        m = ambiguous_mask.reshape(cam.height, cam.width)
        up = [np.where(m, 0.0, u).astype(np.float32) if u.ndim == 2 else
              np.where(m[None], 0.0, u).astype(np.float32) for u in up]
    return up


@pytest.mark.parametrize("tile", [(16, 16), (8, 8), (16, 8), (32, 8)])
def test_backward_matches_oracle_tiny(tile):
    # the backward replays the records each 8x4 block blended in the forward:
    # every tile size (2, 4 or 8 blocks per tile) must give the oracle's gradients
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams(tile_w=tile[0], tile_h=tile[1])
    op = oracle_params(p)
    ref_f = oracle.render(sc, cam, op)
    amb = ref_f["margin"] < AMBIG_MARGIN
    up = _upstream(cam, 7, amb)
    pg, g2, sp, s2 = oracle_grads_with_spread(sc, cam, up, op)
    fr = _frame(sc, cam, p)
    ups = [torch.from_numpy(u).to(DEV) for u in up]
    grads = fr.backward(*ups)[0]
    torch.cuda.synchronize()
    # per-Gaussian 2D gradients (from the sums the compositing backward accumulates)
    dbg = fr.debug()["grad2d"].cpu().numpy()
    v = ref_f["dec"]["valid"]
    rec = grad2d_to_record(dbg[v], {k: ref_f["pre"][k][v] for k in ("conic", "p", "opacity")})
    g2_gpu = {k: rec[k].reshape(g2[k][v].shape) for k in rec}
    g2_ref = {k: g2[k][v] for k in rec}
    assert_grads_close(g2_gpu, g2_ref, {k: s2[k][v] for k in rec}, what="2D gradients")
    gpu = {k: g.cpu().numpy() for k, g in grads.items()}
    assert_grads_close(gpu, pg, sp, what="parameter gradients")


def _clamp_scene():
    """The tiny scene plus large splats centred beyond each border of the image
    widened by the J clamp's margin (and beyond two corners), whose footprints
    still reach the image: their J rows are clamped (3D GS default, Sec. 4.1.1)."""
    sc = scenes.tiny_scene(600, seed=11)
    z = np.array([3.0, 3.5, 2.5, 4.0, 3.2, 2.8], np.float32)
    txy = np.array([[1.2, 0.1], [-1.15, -0.2], [0.2, 1.1], [-0.1, -0.95], [1.1, 1.05], [-1.1, 1.2]], np.float32)
    means = np.c_[txy * z[:, None], z].astype(np.float32)
    rng = np.random.default_rng(12)
    big = scenes.Scene(means, rng.uniform(0.5, 0.9, (6, 3)).astype(np.float32),
                       rng.standard_normal((6, 4)).astype(np.float32),
                       rng.uniform(0.5, 0.95, 6).astype(np.float32),
                       rng.normal(0, 0.3, (6, 1, 3)).astype(np.float32), 0)
    cat = lambda a, b: np.concatenate([a, b]).astype(np.float32)
    return scenes.Scene(cat(sc.means, big.means), cat(sc.scales, big.scales), cat(sc.quats, big.quats),
                        cat(sc.opacities, big.opacities), cat(sc.sh, big.sh), 0), 6


def test_clamped_jacobian_splats_match_oracle():
    # splats whose J clamps: maps over the whole image and per-entry gradients
    sc, n_big = _clamp_scene()
    cam = scenes.tiny_camera()
    p = RenderParams()
    op = oracle_params(p)
    ref_f = oracle.render(sc, cam, op)
    from oracle.params import clamp_limits_f32
    lims = clamp_limits_f32(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, op.clamp_margin)
    tx = (ref_f["pre"]["u"] - cam.cx) / cam.fx
    ty = (ref_f["pre"]["v"] - cam.cy) / cam.fy
    clamped = (tx < lims[0]) | (tx > lims[1]) | (ty < lims[2]) | (ty > lims[3])
    assert (clamped & ref_f["dec"]["valid"])[-n_big:].all()
    fr = _frame(sc, cam, p)
    pixels = np.arange(cam.width * cam.height)
    bad, rep = compare_maps(gpu_maps_at(fr, pixels), ref_f, ref_f["margin"])
    assert rep["ambiguous"] < 1e-2 and rep["n_bad"] == 0, rep
    # the big splats decide what the border pixels show
    a_big = oracle.render(sc.subset(np.arange(sc.n - n_big, sc.n)), cam, op)["alpha"]
    assert (a_big > 0.05).mean() > 0.1
    up = _upstream(cam, 8, ref_f["margin"] < AMBIG_MARGIN)
    pg, _, sp, _ = oracle_grads_with_spread(sc, cam, up, op)
    grads = fr.backward(*[torch.from_numpy(u).to(DEV) for u in up])[0]
    torch.cuda.synchronize()
    gpu = {k: g.cpu().numpy() for k, g in grads.items()}
    assert_grads_close(gpu, pg, sp, what="parameter gradients")
    # the clamped splats' own gradients, at the strict relative bound where FP32 can meet it
    big = {k: v[-n_big:] for k, v in gpu.items()}
    assert_grads_close(big, {k: v[-n_big:] for k, v in pg.items()}, {k: v[-n_big:] for k, v in sp.items()},
                       what="clamped splats' gradients")
    assert all(np.abs(pg[k][-n_big:]).max() > 0 for k in pg)


def test_backward_run_to_run_differences_are_bounded():
    # The compositing backward adds each visit's per-splat sums to the entry's
    # 2D-gradient slots with FP32 atomics, so the order of those additions, and
    # with it the last bits of a gradient, changes from run to run (the
    # per-visit partial sums themselves are computed the same way every time).
    # Stated bound: two runs differ, entry by entry, by at most 1e-5 of the
    # entry plus 8 times its FP32 spread (measured: at most 3.1 times the
    # spread on this scene, under 1 on crops of the 3M scene, and a few ulps
    # on well-conditioned entries); the maps are bit-identical.
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams()
    op = oracle_params(p)
    ref_f = oracle.render(sc, cam, op)
    up = _upstream(cam, 7, ref_f["margin"] < AMBIG_MARGIN)
    fr = _frame(sc, cam, p)
    runs = []
    for _ in range(4):
        g = fr.backward(*[torch.from_numpy(u).to(DEV) for u in up])[0]
        torch.cuda.synchronize()
        runs.append({k: v.cpu().numpy() for k, v in g.items()})
    pg, _, sp, _ = oracle_grads_with_spread(sc, cam, up, op)
    same = 0
    for r in runs[1:]:
        assert_grads_close(r, runs[0], sp, rel=1e-5, c_spread=8.0, what="run-to-run")
        same += sum(int((r[k] == runs[0][k]).sum()) for k in r)
    total = 3 * sum(v.size for v in runs[0].values())
    assert same > 0.5 * total   # most entries come out bit-identical
    fr2 = _frame(sc, cam, p)
    for a, b in zip(fr.view_maps(0), fr2.view_maps(0)):
        torch.testing.assert_close(a, b, rtol=0, atol=0)


def test_forward_after_backward_reports_no_backward_evaluations():
    # every gs_preprocess clears the backward's counters as well as the header's,
    # so gs_check after a forward-only frame does not report an older backward
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    fr = _frame(sc, cam, RenderParams())
    fr.backward(*[torch.from_numpy(u[0]).to(DEV) for u in scenes.upstream_grads(3, cam.height, cam.width)])
    assert fr.stats().n_evals_bwd > 0
    fr.forward()
    st = fr.stats()
    assert st.n_evals_bwd == 0 and st.n_evals_fwd > 0 and st.status == 0


@pytest.mark.parametrize("losses, geo", [(False, False), (True, False), (False, True)])
def test_maps_do_not_depend_on_the_batch(losses, geo):
    # Gaussians per batch (records a warp stages per round: 32 or 64) is a
    # performance knob: bit-identical maps and blend masks, on short (tiny) and
    # long (200K object scene) tile lists, for the plain, the Eq. 23-24 and the
    # geometry-only forward
    for sc, cam in ((scenes.tiny_scene(), scenes.tiny_camera()),
                    (scenes.object_scene(200_000, seed=1), scenes.object_camera(400, 300, 550.0))):
        outs = []
        for batch in (32, 64):
            fr = _frame(sc, cam, RenderParams(batch=batch, losses=losses, geometry_only=geo))
            o = [t.cpu().numpy() for t in fr.view_maps(0) if t is not None]
            if losses:
                o += [t.cpu().numpy() for t in fr.loss_maps(0)]
            st = fr.stats()
            o.append(np.array([st.n_evals_fwd, st.n_blended, st.n_pairs]))
            outs.append(o)
        for a, b in zip(*outs):
            np.testing.assert_array_equal(a, b)


def test_backward_with_batch_64_matches_oracle():
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams(batch=64, tile_w=32, tile_h=8)
    op = oracle_params(p)
    ref_f = oracle.render(sc, cam, op)
    up = _upstream(cam, 9, ref_f["margin"] < AMBIG_MARGIN)
    pg, _, sp, _ = oracle_grads_with_spread(sc, cam, up, op)
    fr = _frame(sc, cam, p)
    g = fr.backward(*[torch.from_numpy(u).to(DEV) for u in up])[0]
    torch.cuda.synchronize()
    assert_grads_close({k: v.cpu().numpy() for k, v in g.items()}, pg, sp, what="batch 64")
