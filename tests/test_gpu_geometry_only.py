"""Forward-only geometry render (alpha, depth, normal; no colour, no backward
state) for fusing many views: identical to the full render's maps, and the
same against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes
from tests._util import AMBIG_MARGIN, TOL_ABS, TOL_DEPTH_REL, oracle_params

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _render(scs, views, p):
    fr = Frame([SceneTensors.from_scene(s, DEV) for s in scs], views, p)
    fr.forward()
    torch.cuda.synchronize()
    assert fr.last_status == 0
    return fr


@pytest.mark.parametrize("tile", [(16, 16), (8, 8)])
def test_geometry_maps_equal_the_full_render(tile):
    sc = scenes.object_scene(60_000, seed=21)
    cam = scenes.object_camera(403, 301, 550.0)
    full = _render([sc], [(cam, 0)], RenderParams(tile_w=tile[0], tile_h=tile[1]))
    geo = _render([sc], [(cam, 0)], RenderParams(tile_w=tile[0], tile_h=tile[1], geometry_only=True))
    c, a, d, n = geo.view_maps(0)
    assert c is None and geo.color is None
    for x, y in zip((a, d, n), full.view_maps(0)[1:]):
        torch.testing.assert_close(x, y, rtol=0, atol=0)
    assert geo.stats().n_pairs == full.stats().n_pairs
    assert geo.stats().n_evals_fwd == full.stats().n_evals_fwd


def test_geometry_maps_match_the_oracle():
    sc, cam = scenes.tiny_scene(seed=7), scenes.tiny_camera()
    p = RenderParams(geometry_only=True)
    fr = _render([sc], [(cam, 0)], p)
    ref = oracle.render(sc, cam, oracle_params(p))
    ok = ref["margin"] >= AMBIG_MARGIN
    _, a, d, n = [None if t is None else t.cpu().numpy() for t in fr.view_maps(0)]
    a, d, n = a.reshape(-1), d.reshape(-1), n.reshape(3, -1).T
    assert np.abs(a - ref["alpha"])[ok].max() <= TOL_ABS
    assert np.abs(n - ref["normal"]).max(1)[ok].max() <= TOL_ABS
    rel = np.abs(d - ref["depth"]) / np.maximum(np.abs(ref["depth"]), 1e-6)
    assert rel[ok].max() <= TOL_DEPTH_REL


def test_many_views_in_one_frame_equal_single_views():
    sc = scenes.object_scene(40_000, seed=22)
    cams = scenes.fusion_cameras(6, seed=3, radius=4.0, width=320, height=208)
    p = RenderParams(geometry_only=True)
    fr = _render([sc], [(c, 0) for c in cams], p)
    for v, c in enumerate(cams):
        one = _render([sc], [(c, 0)], p)
        for x, y in zip(fr.view_maps(v)[1:], one.view_maps(0)[1:]):
            torch.testing.assert_close(x, y, rtol=0, atol=0)
