"""Mip-Splatting 3D filter on the GPU: the variance from the cameras, and the
filtered render and gradients, against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import binning, filter3d
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes
from tests._util import assert_grads_close, oracle_grads_with_spread, AMBIG_MARGIN, _same_ranges, compare_maps, gpu_maps_at, oracle_params

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _bound_distance(means, cams, margin=0.15):
    """Per point, the smallest distance (px, or depth units for z) of any view's
    decision to its threshold: points closer than 1e-3 may flip in FP32."""
    m = np.asarray(means, np.float64)
    dmin = np.full(len(m), np.inf)
    for c in cams:
        V = c.viewmat
        x = m @ V[:3, :3].T + V[:3, 3]
        z = x[:, 2]
        with np.errstate(all="ignore"):
            u = c.fx * x[:, 0] / z + c.cx
            v = c.fy * x[:, 1] / z + c.cy
        d = np.minimum.reduce([np.abs(z - c.near), np.abs(u + margin * c.width),
                               np.abs(u - (1 + margin) * c.width), np.abs(v + margin * c.height),
                               np.abs(v - (1 + margin) * c.height)])
        dmin = np.minimum(dmin, np.nan_to_num(d, nan=0.0))
    return dmin


def test_filter_variance_matches_oracle():
    sc = scenes.object_scene(20_000, seed=31)
    rng = np.random.default_rng(3)
    far = np.c_[rng.uniform(-1, 1, 500), rng.uniform(-40, -25, 500), rng.uniform(-1, 1, 500)]   # overhead
    sc.means = np.ascontiguousarray(np.r_[sc.means[:-500], far], np.float32)
    cams = scenes.fusion_cameras(6, seed=2, radius=4.0, width=320, height=240)
    st = SceneTensors.from_scene(sc, DEV)
    fr = Frame([st], [(c, 0) for c in cams], RenderParams())
    got = fr.filter3d(0, 0.2, attach=False)
    torch.cuda.synchronize()
    got = got.cpu().numpy().astype(np.float64)
    ref, seen = filter3d.filter_variance(sc.means.astype(np.float64), cams)
    assert 0 < seen.sum() < sc.n
    sure = _bound_distance(sc.means, cams) > 1e-3
    fill = ref[~seen].max()
    ok = sure & (seen | (ref[seen][sure[seen]].max() == fill))
    assert ok.mean() > 0.99
    np.testing.assert_allclose(got[ok], ref[ok], rtol=2e-6)


def _filtered_tiny(seed):
    sc = scenes.tiny_scene(seed=seed)
    rng = np.random.default_rng(seed)
    sc.filter_var = rng.uniform(0.0, 1e-3, sc.n).astype(np.float32)   # s^2 ~ 2.5e-3
    return sc


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_filtered_tile_lists_are_bit_exact(tile):
    sc, cam = _filtered_tiny(1), scenes.tiny_camera()
    p = RenderParams(tile_w=tile[0], tile_h=tile[1])
    fr = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p)
    fr.forward()
    dbg = fr.debug()
    op = oracle_params(p)
    dec = binning.decide_scene(sc, cam, op)
    tile_ref, g_ref, ranges_ref = binning.tile_lists(dec, cam, op)
    np.testing.assert_array_equal(dbg["pair_tile"].cpu().numpy(), tile_ref)
    np.testing.assert_array_equal(dbg["pair_entry"].cpu().numpy(), g_ref)
    _same_ranges(dbg["ranges"].cpu().numpy(), ranges_ref)
    # the filter changes the lists (it widens every splat)
    plain = binning.decide(sc.means, sc.scales, sc.quats, sc.opacities, cam, op)
    assert (plain["rect"] != dec["rect"]).any()


def test_filtered_maps_and_gradients_match_oracle():
    sc, cam = _filtered_tiny(2), scenes.tiny_camera()
    p = RenderParams()
    op = oracle_params(p)
    fr = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p)
    fr.forward()
    torch.cuda.synchronize()
    ref = oracle.render(sc, cam, op)
    bad, rep = compare_maps(gpu_maps_at(fr, np.arange(cam.width * cam.height)), ref, ref["margin"])
    assert rep["n_bad"] == 0 and rep["ambiguous"] < 1e-2, rep
    amb = (ref["margin"] < AMBIG_MARGIN).reshape(cam.height, cam.width)
    up = [u[0] for u in scenes.upstream_grads(9, cam.height, cam.width)]
    up = [np.where(amb if u.ndim == 2 else amb[None], 0.0, u).astype(np.float32) for u in up]
    pg, _, sp, _ = oracle_grads_with_spread(sc, cam, up, op)
    g = fr.backward(*[torch.from_numpy(u).to(DEV) for u in up])[0]
    torch.cuda.synchronize()
    assert_grads_close({k: v.cpu().numpy() for k, v in g.items()}, pg, sp, what="filtered gradients")
