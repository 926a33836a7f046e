"""Depth ties across several radix-sort blocks: splats whose camera-space
depths are bit-identical must keep the order of their entry index (the sort
key is (tile, depth bits, Gaussian id), Sec. 3's tile-based rasterizer), also
when the equal keys are spread over many one-sweep blocks and every digit of
a pass is shared by a whole warp."""
import numpy as np
import pytest
import torch

import oracle
from oracle import binning
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes
from tests._util import _same_ranges, compare_maps, gpu_maps_at, oracle_params

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _axis_camera():
    # looks down +z with the axes of the world: a camera-space depth is the
    # world z plus zero terms, so equal world z gives bit-equal depths
    return scenes.Camera(scenes.look_at((0.0, 0.0, 0.0), (0.0, 0.0, 1.0)), 220.0, 220.0, 128.0, 96.0, 256, 192)


def _tied_scene(n, depths, seed):
    rng = np.random.default_rng(seed)
    z = np.asarray(depths, np.float32)[rng.integers(0, len(depths), n)]
    means = np.stack([rng.uniform(-0.55, 0.55, n) * z, rng.uniform(-0.42, 0.42, n) * z, z], 1).astype(np.float32)
    scales = rng.uniform(0.004, 0.03, (n, 3)).astype(np.float32)
    q = rng.normal(size=(n, 4)).astype(np.float32)
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = rng.uniform(0.3, 0.9, n).astype(np.float32)
    sh = rng.normal(0.0, 0.5, (n, 4, 3)).astype(np.float32)
    return scenes.Scene(means, scales, q, op, sh, 1)


@pytest.mark.parametrize("depths", [(2.0, 2.5, 3.0), (2.0,)])
def test_equal_depths_keep_index_order_across_sort_blocks(depths):
    sc, cam = _tied_scene(24000, depths, seed=len(depths)), _axis_camera()
    p = RenderParams()
    fr = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p)
    fr.forward()
    torch.cuda.synchronize()
    op = oracle_params(p)
    dec = binning.decide(sc.means, sc.scales, sc.quats, sc.opacities, cam, op)
    zk = dec["zkey"][dec["valid"]]
    assert len(np.unique(zk)) == len(depths)          # the depths are tied bit for bit
    assert dec["valid"].sum() > 3 * 4096              # spread over several sort blocks
    tile_ref, g_ref, ranges_ref = binning.tile_lists(dec, cam, op)
    assert len(tile_ref) > 3 * 4096
    dbg = fr.debug()
    np.testing.assert_array_equal(dbg["pair_tile"].cpu().numpy(), tile_ref)
    np.testing.assert_array_equal(dbg["pair_entry"].cpu().numpy(), g_ref)
    _same_ranges(dbg["ranges"].cpu().numpy(), ranges_ref)
    # the blend order of tied splats shows in the maps: a crop against the oracle
    ys, xs = np.mgrid[80:112, 112:144]
    pix = (ys * cam.width + xs).reshape(-1)
    ref = oracle.render(sc, cam, op, pixels=pix)
    bad, rep = compare_maps(gpu_maps_at(fr, pix), ref, ref["margin"])
    assert rep["n_bad"] == 0 and rep["ambiguous"] <= 0.02, rep
