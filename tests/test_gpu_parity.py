"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tile lists and sort order: bit-exact.  Colour, alpha, normal: 1e-4 absolute;
depth: 1e-4 relative, on pixels whose discrete decisions are not within the
FP32/FP64 ambiguity margin.  Gradients: relative 1e-3 of each parameter
group's scale.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import binning
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes
from tests._util import _same_ranges, AMBIG_MARGIN, compare_maps, gpu_maps_at, grad2d_to_record, oracle_params

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


def _grad_compare(g_gpu, g_ref, rel=1e-3):
    """Per-array check: |gpu - ref| <= rel * max|ref| elementwise, plus a norm check."""
    out = {}
    for k in g_ref:
        a = np.asarray(g_gpu[k], np.float64)
        b = np.asarray(g_ref[k], np.float64)
        scale = np.abs(b).max()
        err = np.abs(a - b).max()
        out[k] = (err / max(scale, 1e-30), np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
    return out


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
    pg, g2, _ = oracle.render_grads(sc, cam, up, op)
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
    rep2 = _grad_compare(g2_gpu, g2_ref)
    for k, (emax, enorm) in rep2.items():
        assert emax < 1e-3 and enorm < 1e-3, (k, rep2)
    gpu = {k: g.cpu().numpy() for k, g in grads.items()}
    rep = _grad_compare(gpu, pg)
    for k, (emax, enorm) in rep.items():
        assert emax < 1e-3 and enorm < 1e-3, (k, rep)
