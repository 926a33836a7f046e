"""The bounds-checked build (libgs_debug.so, -DGS_DEBUG): on every kind of
frame the ordinary tests render, none of its device-side index checks fires,
and it renders the same maps (bit for bit) and the same gradients (within the
run-to-run spread of the atomics) as the ordinary build.  A stand-in for a
memory checker, which is not available to these tests."""
import pytest
import torch

from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, _lib, build, scenes

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.fixture(scope="module")
def libs():
    build.build()
    build.build(debug=True)
    rel, dbg = _lib.load(), _lib.load(_lib.DEBUG_LIB_PATH)
    assert rel.gs_debug_checks() == 0 and dbg.gs_debug_checks() == 1
    return rel, dbg


def _render(lib, scs, views, params, cap=None, backward=True, seed=3):
    sts = [SceneTensors.from_scene(s, DEV) for s in scs]
    fr = Frame(sts, views, params, pair_capacity=cap, lib=lib)
    fr.forward()   # grows the pair capacity if it was too small
    maps = [m.clone() for v in range(len(views)) for m in fr.view_maps(v) if m is not None]
    grads = None
    if backward:   # one seeded upstream per view, concatenated in view order like the maps
        per_view = [scenes.upstream_grads(seed + v, c.height, c.width) for v, (c, _) in enumerate(views)]
        up = [torch.cat([torch.from_numpy(u[k][0]).reshape(-1) for u in per_view]).to(DEV) for k in range(4)]
        grads = fr.backward(*up)
    st = fr.stats()
    assert st.status == 0, _lib.STATUS_NAMES.get(st.status, st.status)
    return maps, grads


def _compare(libs, scs, views, params, **kw):
    rel, dbg = libs
    m0, g0 = _render(rel, scs, views, params, **kw)
    m1, g1 = _render(dbg, scs, views, params, **kw)
    for a, b in zip(m0, m1):
        assert torch.equal(a, b)
    if g0 is not None:
        for d0, d1 in zip(g0, g1):
            for k in d0:
                scale = float(d0[k].abs().max()) + 1e-30
                torch.testing.assert_close(d1[k], d0[k], rtol=1e-3, atol=1e-4 * scale)


@pytest.mark.parametrize("tile", [(16, 16), (32, 8), (8, 8)])
def test_tiny_scene(libs, tile):
    p = RenderParams()
    p.tile_w, p.tile_h = tile
    _compare(libs, [scenes.tiny_scene()], [(scenes.tiny_camera(), 0)], p)


def test_object_scene_ragged_with_losses_and_batch_64(libs):
    p = RenderParams()
    p.batch = 64
    p.losses = True
    cam = scenes.object_camera(125 * 4 + 3, 107 * 3 + 1, 700.0)
    _compare(libs, [scenes.object_scene(200_000, seed=1)], [(cam, 0)], p)


def test_several_views_of_several_scenes(libs):
    scs = [scenes.object_scene(50_000, seed=5), scenes.tiny_scene(3000, seed=2)]
    views = [(scenes.object_camera(320, 240, 400.0), 0), (scenes.object_camera(200, 150, 300.0), 0),
             (scenes.tiny_camera(), 1)]
    _compare(libs, scs, views, RenderParams())


def test_geometry_only(libs):
    p = RenderParams()
    p.geometry_only = True
    _compare(libs, [scenes.object_scene(200_000, seed=1)], [(scenes.object_camera(), 0)], p, backward=False)


def test_capacity_overflow_then_grown(libs):
    _compare(libs, [scenes.tiny_scene()], [(scenes.tiny_camera(), 0)], RenderParams(), cap=100)


def _corrupt_pair_entries(fr, tile, value=-1):
    """Overwrite the entries of one tile's list in the frame's workspace (found
    by matching the sorted pair entries that gs_debug_copy returns)."""
    d = fr.debug()
    pe, rg = d["pair_entry"], d["ranges"]
    base = (fr.ws.data_ptr() + 255) // 256 * 256 - fr.ws.data_ptr()
    words = fr.ws[base:base + (fr.ws.numel() - base) // 4 * 4].view(torch.int32)
    n = pe.numel()
    cand = torch.nonzero(words[: words.numel() - n + 1] == pe[0]).flatten().tolist()
    hits = [c for c in cand if torch.equal(words[c:c + n], pe)]
    assert len(hits) == 1, hits
    lo, hi = int(rg[tile, 0]), int(rg[tile, 1])
    assert hi > lo
    words[hits[0] + lo:hits[0] + hi] = value
    return lo, hi


def _largest_tile(fr):
    rg = fr.debug()["ranges"]
    return int(torch.argmax(rg[:, 1] - rg[:, 0]))


def test_a_corrupted_tile_list_is_caught_by_the_forward(libs):
    _, dbg = libs
    assert dbg.gs_debug_checks() == 1   # never run a corrupted workspace through the ordinary build
    st = SceneTensors.from_scene(scenes.tiny_scene(), DEV)
    fr = Frame([st], [(scenes.tiny_camera(), 0)], RenderParams(), lib=dbg)
    fr.forward()
    assert fr.stats().status == 0
    _corrupt_pair_entries(fr, _largest_tile(fr))
    fr.render()
    fr.stats()
    assert fr.last_status == _lib.GS_ERR_BOUNDS
    msg = dbg.gs_last_error_string().decode()
    assert "compositing forward: tile-list entry" in msg and "4294967295" in msg, msg


def test_a_corrupted_tile_list_is_caught_by_the_backward(libs):
    _, dbg = libs
    assert dbg.gs_debug_checks() == 1
    cam = scenes.tiny_camera()
    st = SceneTensors.from_scene(scenes.tiny_scene(), DEV)
    fr = Frame([st], [(cam, 0)], RenderParams(), lib=dbg)
    fr.forward()
    assert fr.stats().status == 0
    _corrupt_pair_entries(fr, _largest_tile(fr))
    up = [torch.from_numpy(u[0]).to(DEV) for u in scenes.upstream_grads(3, cam.height, cam.width)]
    fr.backward(*up)
    fr.stats()
    assert fr.last_status == _lib.GS_ERR_BOUNDS
    msg = dbg.gs_last_error_string().decode()
    assert "compositing backward: tile-list entry" in msg and "4294967295" in msg, msg
