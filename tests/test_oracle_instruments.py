"""Pins of the oracle's two test instruments (no GPU): the switch that runs its
arithmetic in FP32, and the per-entry FP32 spread of its gradients that the GPU
gradient checks scale their bound with."""
import numpy as np
import torch

import oracle
from oracle import RenderParams
from paper_2406_01467_b300 import scenes


def _small():
    sc = scenes.tiny_scene(60, seed=4)
    cam = scenes.Camera(np.eye(4), 40.0, 40.0, 16.0, 12.0, 32, 24)
    up = [u[0] for u in scenes.upstream_grads(5, 24, 32)]
    return sc, cam, up


def test_fp32_evaluation_rounds_and_restores():
    sc, cam, up = _small()
    prm = RenderParams()
    r64 = oracle.render(sc, cam, prm)
    with oracle.evaluated_in(torch.float32):
        r32 = oracle.render(sc, cam, prm)
        g32 = oracle.render_grads(sc, cam, up, prm)[0]
    assert r32["color"].dtype == np.float32 and g32["means"].dtype == np.float32
    ok = (r64["margin"] > 1e-3) & (r32["margin"] > 1e-3)
    err = np.abs(r32["color"] - r64["color"])[ok].max()
    assert 0 < err < 1e-5            # rounded, and only by FP32 rounding
    again = oracle.render(sc, cam, prm)
    assert again["color"].dtype == np.float64
    np.testing.assert_array_equal(again["color"], r64["color"])   # FP64 restored exactly


def test_spread_moves_inputs_by_at_most_one_ulp():
    # with a "gradient" that is an input itself, FP32 evaluation is exact and the
    # samples at moved inputs change each entry by 0 or exactly one FP32 ulp
    sc, _, _ = _small()
    ref, spread = oracle.fp32_spread(lambda s: {"m": np.asarray(s.means, np.float64)}, sc, samples=4)
    np.testing.assert_array_equal(ref["m"], np.asarray(sc.means, np.float64))
    ulp = np.spacing(np.abs(np.asarray(sc.means, np.float32))).astype(np.float64)
    assert (spread["m"] <= ulp * (1 + 1e-12)).all()
    assert (spread["m"] == 0).mean() < 0.2   # most entries were moved in some sample


def test_spread_bounds_the_fp32_error_and_is_small_where_well_conditioned():
    sc, cam, up = _small()
    prm = RenderParams()
    ref, spread = oracle.fp32_spread(lambda s: oracle.render_grads(s, cam, up, prm)[0], sc)
    pg = oracle.render_grads(sc, cam, up, prm)[0]
    with oracle.evaluated_in(torch.float32):
        g32 = oracle.render_grads(sc, cam, up, prm)[0]
    for k in pg:
        np.testing.assert_array_equal(ref[k], pg[k])
        assert (np.abs(g32[k] - pg[k]) <= spread[k]).all()       # the unmoved sample is included
        big = np.abs(pg[k]) > 1e-2 * np.abs(pg[k]).max()
        assert np.median(spread[k][big] / np.abs(pg[k][big])) < 1e-5   # FP32-level where it is well conditioned
