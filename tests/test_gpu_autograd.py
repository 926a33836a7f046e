"""The differentiable entry point ``rasterize`` (a torch.autograd.Function over
gs_render_fwd / gs_render_bwd) on the GPU.

* its gradients, taken by torch.autograd.grad of a seeded linear loss on all
  four maps, match the FP64 oracle's analytic gradient entry by entry, and
  central finite differences of the FP64 oracle's loss (relative 1e-3);
* a second call on the same workspace with new parameter values renders and
  differentiates those values;
* with a preset pair capacity nothing synchronises, and a whole training step
  (render, loss, gradients) captured in a CUDA graph replays the eager step.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, rasterize, scenes
from tests._util import (AMBIG_MARGIN, assert_grads_close, compare_maps, gpu_maps_at, oracle_grads_with_spread,
                         oracle_params)

pytestmark = pytest.mark.gpu
DEV = "cuda"
NAMES = ("means", "scales", "quats", "opacities", "sh")


def _leaves(sc, dtype=torch.float32):
    return [torch.tensor(np.asarray(getattr(sc, k)), dtype=dtype, device=DEV, requires_grad=True) for k in NAMES]


def _loss(outs, up):
    return sum((o * u).sum() for o, u in zip(outs, up))


def _upstream(cam, seed, amb):
    m = amb.reshape(cam.height, cam.width)
    up = [u[0] for u in scenes.upstream_grads(seed, cam.height, cam.width)]
    return [np.where(m if u.ndim == 2 else m[None], 0.0, u).astype(np.float32) for u in up]


def _fd_loss(sc, cam, op, up, sel, pix):
    """The loss restricted to pixels ``pix`` with the Gaussians ``sel`` (every
    Gaussian that can reach them), in FP64."""
    r = oracle.render(sc.subset(sel), cam, op, pixels=pix)
    dC, dA, dD, dN = [np.asarray(u, np.float64) for u in up]
    return float((r["color"] * dC.reshape(3, -1)[:, pix].T).sum() + (r["alpha"] * dA.reshape(-1)[pix]).sum()
                 + (r["depth"] * dD.reshape(-1)[pix]).sum() + (r["normal"] * dN.reshape(3, -1)[:, pix].T).sum())


def test_rasterize_gradients_match_oracle_and_finite_differences():
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams()
    op = oracle_params(p)
    ref = oracle.render(sc, cam, op)
    up = _upstream(cam, 21, ref["margin"] < AMBIG_MARGIN)
    leaves = _leaves(sc)
    outs = rasterize(*leaves, cam, sc.sh_degree, p)
    assert [tuple(o.shape) for o in outs] == [(3, 128, 128), (128, 128), (128, 128), (3, 128, 128)]
    grads = torch.autograd.grad(_loss(outs, [torch.from_numpy(u).to(DEV) for u in up]), leaves)
    gpu = {k: g.detach().cpu().numpy() for k, g in zip(NAMES, grads)}
    pg, _, sp, _ = oracle_grads_with_spread(sc, cam, up, op)
    assert_grads_close(gpu, pg, sp, what="rasterize vs oracle")

    # central differences of the FP64 oracle's loss on a sample of parameters of
    # Gaussians with large gradients; only the pixels of the perturbed Gaussian's
    # rectangle change, so the loss is taken there, over the Gaussians reaching them
    dec = ref["dec"]
    rect = dec["rect"]
    rng = np.random.default_rng(5)
    zs = np.asarray(sc.means, np.float64)   # depth ties within 1e-5 could swap order under a step
    checked = 0
    for name in NAMES:
        g = gpu[name].reshape(sc.n, -1)
        mag = np.abs(g).max(1)
        cand = np.nonzero(dec["valid"] & (mag > 1e-2 * mag.max()))[0]
        for gi in rng.choice(cand, 5, replace=False):
            i0, i1, j0, j1 = rect[gi]
            ys, xs = np.mgrid[j0:j1 + 1, i0:i1 + 1]
            pix = (ys * cam.width + xs).reshape(-1)
            sel = np.nonzero(dec["valid"] & (rect[:, 1] >= i0) & (rect[:, 0] <= i1)
                             & (rect[:, 3] >= j0) & (rect[:, 2] <= j1))[0]
            others = sel[sel != gi]
            if len(others) and np.abs(zs[others, 2] / zs[gi, 2] - 1).min() < 1e-5:
                continue
            comp = int(np.argmax(np.abs(g[gi])))
            base = np.asarray(getattr(sc, name), np.float64)
            flat = base.reshape(sc.n, -1)
            h = 1e-6 * max(1.0, abs(flat[gi, comp]))
            vals = []
            for sgn in (1, -1):
                mod = flat.copy()
                mod[gi, comp] += sgn * h
                s2 = scenes.Scene(**{**sc.__dict__, name: mod.reshape(base.shape)})
                vals.append(_fd_loss(s2, cam, op, up, sel, pix))
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(g[gi, comp] - fd) <= 1e-3 * abs(fd), (name, gi, comp, g[gi, comp], fd)
            checked += 1
    assert checked >= 20


def test_rasterize_reuses_its_frame_with_new_values():
    sc, cam = scenes.tiny_scene(1200, seed=3), scenes.tiny_camera()
    p = RenderParams()
    op = oracle_params(p)
    l1 = _leaves(sc)
    up1 = _upstream(cam, 4, oracle.render(sc, cam, op)["margin"] < AMBIG_MARGIN)
    o1 = rasterize(*l1, cam, sc.sh_degree, p)
    fr = o1[0].grad_fn.frame
    g1 = torch.autograd.grad(_loss(o1, [torch.from_numpy(u).to(DEV) for u in up1]), l1)
    rng = np.random.default_rng(9)
    sc2 = sc.subset(np.arange(sc.n))
    sc2.means = (sc.means + 0.02 * rng.standard_normal(sc.means.shape)).astype(np.float32)
    sc2.opacities = np.clip(sc.opacities * rng.uniform(0.7, 1.1, sc.n), 0.01, 0.99).astype(np.float32)
    ref2 = oracle.render(sc2, cam, op)
    up2 = _upstream(cam, 4, ref2["margin"] < AMBIG_MARGIN)
    l2 = _leaves(sc2)
    o2 = rasterize(*l2, cam, sc.sh_degree, p, frame=fr)
    assert o2[0].grad_fn.frame is fr
    g2 = torch.autograd.grad(_loss(o2, [torch.from_numpy(u).to(DEV) for u in up2]), l2)
    # the second call renders and differentiates the new values
    bad, rep = compare_maps(gpu_maps_at(fr, np.arange(cam.width * cam.height)), ref2, ref2["margin"])
    assert rep["n_bad"] == 0, rep
    for a, b in zip(o2, fr.view_maps(0)):
        torch.testing.assert_close(a, b, rtol=0, atol=0)
    pg, _, sp, _ = oracle_grads_with_spread(sc2, cam, up2, op)
    assert_grads_close({k: g.cpu().numpy() for k, g in zip(NAMES, g2)}, pg, sp, what="second call vs oracle")
    assert (o1[1] - o2[1]).abs().max().item() > 1e-2
    assert (g1[0] - g2[0]).abs().max().item() > 1e-3 * g2[0].abs().max().item()


def test_rasterize_training_step_in_a_cuda_graph():
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams()
    op = oracle_params(p)
    up_np = [u[0] for u in scenes.upstream_grads(6, cam.height, cam.width)]
    up = [torch.from_numpy(u).to(DEV) for u in up_np]   # captured: refilled before every replay
    leaves = _leaves(sc)
    probe = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p)
    probe.forward()
    cap = int(probe.stats().n_pairs * 2)
    fr = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p, pair_capacity=cap)

    def step():
        outs = rasterize(*leaves, cam, sc.sh_degree, p, pair_capacity=cap, frame=fr)
        return outs, torch.autograd.grad(_loss(outs, up), leaves)

    torch.autograd.graph.set_warn_on_accumulate_grad_stream_mismatch(False)   # leaves outlive the warm-up graphs
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(2):
            step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        s_outs, s_grads = step()
    rng = np.random.default_rng(2)
    for it in range(2):
        # new values in the captured parameter and upstream tensors
        sc_it = sc.subset(np.arange(sc.n))
        sc_it.means = (sc.means + 0.01 * rng.standard_normal(sc.means.shape)).astype(np.float32)
        sc_it.opacities = (sc.opacities * rng.uniform(0.8, 1.0, sc.n)).astype(np.float32)
        ref = oracle.render(sc_it, cam, op)
        up_it = _upstream(cam, 6, ref["margin"] < AMBIG_MARGIN)
        with torch.no_grad():
            leaves[0].copy_(torch.from_numpy(sc_it.means))
            leaves[3].copy_(torch.from_numpy(sc_it.opacities))
            for u, v in zip(up, up_it):
                u.copy_(torch.from_numpy(v))
        graph.replay()
        torch.cuda.synchronize()
        assert fr.stats().status == 0
        bad, rep = compare_maps(gpu_maps_at(fr, np.arange(cam.width * cam.height)), ref, ref["margin"])
        assert rep["n_bad"] == 0, rep
        pg, _, sp, _ = oracle_grads_with_spread(sc_it, cam, up_it, op)
        assert_grads_close({k: g.cpu().numpy() for k, g in zip(NAMES, s_grads)}, pg, sp,
                           what=f"graph replay {it} vs oracle")
        e_outs, e_grads = step()   # the eager step on the same values renders the same maps
        torch.cuda.synchronize()
        for a, b in zip(s_outs, e_outs):
            torch.testing.assert_close(a, b, rtol=0, atol=0)


def test_rasterize_bf16_parameters_give_bf16_gradients():
    sc, cam = scenes.tiny_scene(1000, seed=7), scenes.tiny_camera()
    p = RenderParams()
    up = [torch.from_numpy(u[0]).to(DEV) for u in scenes.upstream_grads(8, cam.height, cam.width)]
    lb = _leaves(sc, torch.bfloat16)
    ob = rasterize(*lb, cam, sc.sh_degree, p)
    gb = torch.autograd.grad(_loss(ob, up), lb)
    assert all(g.dtype == torch.bfloat16 for g in gb)
    r = scenes.to_bf16_rounded
    sc_r = scenes.Scene(r(sc.means), r(sc.scales), r(sc.quats), r(sc.opacities), r(sc.sh), sc.sh_degree)
    lf = _leaves(sc_r)
    of = rasterize(*lf, cam, sc.sh_degree, p)
    gf = torch.autograd.grad(_loss(of, up), lf)
    for a, b in zip(ob, of):   # the same FP32 compositing after widening
        torch.testing.assert_close(a, b, rtol=0, atol=0)
    for a, b in zip(gb, gf):   # FP32 gradients rounded once to BF16
        torch.testing.assert_close(a.float(), b.to(torch.bfloat16).float(), rtol=1e-2, atol=1e-5 * b.abs().max().item())


def test_rasterize_without_sync_reports_a_capacity_overflow():
    """With a preset pair capacity below the frame's need, nothing synchronises:
    the compositing kernels skip the frame (its maps are left unwritten and
    its 2D gradients stay zero, so the parameter gradients come out zero), the
    frame reports GS_ERR_CAPACITY and the pairs it needed, and a frame of that
    size then renders and differentiates like the synchronising call."""
    from paper_2406_01467_b300 import _lib
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    p = RenderParams()
    up = [torch.from_numpy(u[0]).to(DEV) for u in scenes.upstream_grads(8, cam.height, cam.width)]
    leaves = _leaves(sc)
    small = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p, pair_capacity=64)
    outs = rasterize(*leaves, cam, sc.sh_degree, p, pair_capacity=64, frame=small)
    grads = torch.autograd.grad(_loss(outs, up), leaves)
    torch.cuda.synchronize()
    st = small.stats()
    assert small.last_status == _lib.GS_ERR_CAPACITY and st.n_pairs > 64
    assert all(bool((g == 0).all()) for g in grads)
    need = int(st.n_pairs)
    big = Frame([SceneTensors.from_scene(sc, DEV)], [(cam, 0)], p, pair_capacity=need)
    outs_b = rasterize(*leaves, cam, sc.sh_degree, p, pair_capacity=need, frame=big)
    grads_b = torch.autograd.grad(_loss(outs_b, up), leaves)
    torch.cuda.synchronize()
    assert big.stats().status == 0
    outs_s = rasterize(*leaves, cam, sc.sh_degree, p)   # synchronising, grown as needed
    grads_s = torch.autograd.grad(_loss(outs_s, up), leaves)
    for a, b in zip(outs_b, outs_s):
        torch.testing.assert_close(a, b, rtol=0, atol=0)   # the forward is deterministic
    for a, b in zip(grads_b, grads_s):   # the backward's atomics add in any order
        torch.testing.assert_close(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max()))
