"""CUDA-graph capture of a whole forward + backward step, the tile autotuner, and
the BF16-storage accuracy on the 3M-Gaussian frame (error against the FP64
oracle on a central 128x128 crop)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, autotune, scenes
from tests._util import AMBIG_MARGIN, compare_maps, gpu_maps_at, oracle_params

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _setup(sc, cam, p=None, dtype=torch.float32):
    st = SceneTensors.from_scene(sc, DEV, dtype)
    fr = Frame([st], [(cam, 0)], p or RenderParams())
    fr.forward()
    fr._alloc(int(fr.stats().n_pairs * 1.25) + 1024)
    up = [torch.from_numpy(u[0]).to(DEV) for u in scenes.upstream_grads(3, cam.height, cam.width)]
    return fr, up


def test_graph_replay_matches_eager_step():
    sc, cam = scenes.object_scene(30_000, seed=9), scenes.object_camera(400, 300, 550.0)
    fr, up = _setup(sc, cam)
    grads = fr.alloc_grads()
    step = autotune.make_step(fr, up, grads)
    step()
    torch.cuda.synchronize()
    maps0 = [t.clone() for t in fr.view_maps(0)]
    g0 = {k: v.clone() for k, v in grads[0].items()}
    graph = autotune.capture(step)
    for _ in range(2):
        for t in list(fr.view_maps(0)) + list(grads[0].values()):
            t.zero_()
        graph.replay()
        torch.cuda.synchronize()
        for a, b in zip(fr.view_maps(0), maps0):
            torch.testing.assert_close(a, b, rtol=0, atol=0)
        for k in g0:   # float atomics: equal up to summation order
            torch.testing.assert_close(grads[0][k], g0[k], rtol=1e-4, atol=1e-6 * g0[k].abs().max().item())
    assert fr.stats().status == 0


def test_autotuner_returns_a_candidate_and_caches_it(tmp_path):
    sc, cam = scenes.object_scene(20_000, seed=10), scenes.object_camera(320, 240, 440.0)
    st = SceneTensors.from_scene(sc, DEV)
    cache = str(tmp_path / "tiles.json")
    cands = ((16, 16), (8, 8), (16, 8))
    p, rep = autotune.tune_tile([st], [(cam, 0)], RenderParams(), candidates=cands, iters=2, cache_path=cache)
    # every (tile, Gaussians-per-batch) pair is timed
    assert (p.tile_w, p.tile_h) in cands and p.batch in (32, 64) and not rep["cached"]
    assert sorted(rep["all"]) == sorted(f"{w}x{h}/b{b}" for w, h in cands for b in (32, 64))
    p2, rep2 = autotune.tune_tile([st], [(cam, 0)], RenderParams(), candidates=cands, cache_path=cache)
    assert rep2["cached"] and (p2.tile_w, p2.tile_h, p2.batch) == (p.tile_w, p.tile_h, p.batch)


@pytest.mark.slow
def test_bf16_storage_error_on_central_crop():
    # The 3M / 1297x840 frame with BF16 parameters.  (i) against the oracle fed
    # the same BF16-rounded parameters: compute precision, FP32 tolerances;
    # (ii) against the oracle fed the FP32 parameters: storage quantisation,
    # reported (BF16's 8-bit mantissa moves far splats by decimetres).
    sc, cam = scenes.unbounded_scene(), scenes.unbounded_camera()
    p = RenderParams()
    fr, _ = _setup(sc, cam, p, torch.bfloat16)
    ys, xs = np.mgrid[356:484, 584:712]
    pix = (ys * cam.width + xs).reshape(-1)
    r = scenes.to_bf16_rounded
    sc_r = scenes.Scene(r(sc.means), r(sc.scales), r(sc.quats), r(sc.opacities), r(sc.sh), sc.sh_degree)
    op = oracle_params(p)
    gpu = gpu_maps_at(fr, pix)

    def near_crop(s):   # the Gaussians whose rectangles reach the crop (same order)
        from oracle import binning
        d = binning.decide(s.means, s.scales, s.quats, s.opacities, cam, op)
        rc = d["rect"]
        sel = d["valid"] & (rc[:, 1] >= 584) & (rc[:, 0] <= 711) & (rc[:, 3] >= 356) & (rc[:, 2] <= 483)
        return s.subset(np.nonzero(sel)[0])

    ref_r = oracle.render(near_crop(sc_r), cam, op, pixels=pix)
    bad, rep = compare_maps(gpu, ref_r, ref_r["margin"])
    assert rep["n_bad"] == 0, rep
    ref_f = oracle.render(near_crop(sc), cam, op, pixels=pix)
    errs = {k: float(np.abs(g - ref_f[k]).max()) for g, k in zip(gpu, ("color", "alpha", "depth", "normal"))}
    print("bf16 compute error (same rounded inputs):", rep)
    print("bf16 storage error (fp32 inputs):", errs)
    assert all(np.isfinite(v) for v in errs.values())


def test_bf16_filtered_losses_multiview_matches_fp32_on_rounded_inputs():
    # every option at once: BF16 storage, 3D filter, loss maps, two views of two
    # scenes; against the FP32 path fed the same BF16-rounded parameters
    r = scenes.to_bf16_rounded
    rng = np.random.default_rng(4)
    scs = []
    for seed in (5, 6):
        s = scenes.object_scene(20_000, seed=seed)
        s = scenes.Scene(r(s.means), r(s.scales), r(s.quats), r(s.opacities), r(s.sh), s.sh_degree)
        s.filter_var = rng.uniform(0.0, 1e-5, s.n).astype(np.float32)
        scs.append(s)
    views = [(scenes.object_camera(257, 193, 330.0), 0), (scenes.object_camera(240, 176, 300.0), 1)]
    p = RenderParams(losses=True)
    outs = []
    for dt in (torch.bfloat16, torch.float32):
        fr = Frame([SceneTensors.from_scene(s, DEV, dt) for s in scs], views, p)
        fr.forward()
        ups = [torch.randn(k * fr.n_pixels, device=DEV, generator=torch.Generator(device=DEV).manual_seed(k))
               for k in (3, 1, 1, 3, 1, 1)]
        g = fr.backward(*ups[:4], ddist=ups[4], dnloss=ups[5])
        torch.cuda.synchronize()
        assert fr.stats().status == 0
        outs.append(([t.clone() for v in range(2) for t in fr.view_maps(v) + fr.loss_maps(v)], g))
    for a, b in zip(outs[0][0], outs[1][0]):
        torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-4)
    for ga, gb in zip(outs[0][1], outs[1][1]):
        for k in ga:
            s_ = gb[k].abs().max().item()
            assert (ga[k] - gb[k]).abs().max().item() <= 1e-3 * s_ + 1e-12, k
