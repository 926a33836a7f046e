"""Pins of the oracle's depth distortion (Eq. 23) and normal consistency (Eq. 24)."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import losses
from oracle import RenderParams
from paper_2406_01467_b300 import scenes

DT = torch.float64


def test_distortion_of_two_splats_is_closed_form():
    # two weights w1, w2 at depths d1, d2: sum over ordered pairs = 2 w1 w2 (d1 - d2)^2
    w = torch.tensor([[0.3, 0.45, 0.0]], dtype=DT)
    d = torch.tensor([[2.0, 3.5, 9.0]], dtype=DT)
    ref = 2 * 0.3 * 0.45 * 1.5 ** 2
    assert abs(losses.depth_distortion(w, d).item() - ref) < 1e-14
    assert abs(losses.depth_distortion_pairwise(w, d).item() - ref) < 1e-14


def test_distortion_expansion_equals_double_sum():
    rng = np.random.default_rng(0)
    w = torch.tensor(rng.uniform(0, 0.2, (50, 12)), dtype=DT)
    d = torch.tensor(rng.uniform(1, 5, (50, 12)), dtype=DT)
    np.testing.assert_allclose(losses.depth_distortion(w, d).numpy(),
                               losses.depth_distortion_pairwise(w, d).numpy(), rtol=1e-12)


def test_distortion_gradient_treats_weights_as_constants():
    w = torch.tensor([[0.3, 0.45, 0.1]], dtype=DT, requires_grad=True)
    d = torch.tensor([[2.0, 3.5, 2.5]], dtype=DT, requires_grad=True)
    L = losses.depth_distortion(w, d).sum()
    gw, gd = torch.autograd.grad(L, [w, d], allow_unused=True)
    assert gw is None or torch.count_nonzero(gw) == 0
    W, S1 = w.sum(), (w * d).sum()
    np.testing.assert_allclose(gd.numpy(), (4 * w * (d * W - S1)).detach().numpy(), rtol=1e-13)


def _plane_depth(n, h, cam):
    """Depth map of the plane n . P = h seen by ``cam`` (camera frame)."""
    ii = np.arange(cam.width) + 0.5
    jj = np.arange(cam.height) + 0.5
    rx = ((ii - cam.cx) / cam.fx)[None, :]
    ry = ((jj - cam.cy) / cam.fy)[:, None]
    return h / (n[0] * rx + n[1] * ry + n[2])


@pytest.mark.parametrize("n", [(0.0, 0.0, -1.0), (0.3, -0.2, -0.9), (-0.5, 0.4, -0.7)])
def test_depth_map_normal_of_a_plane_is_its_normal(n):
    n = np.asarray(n) / np.linalg.norm(n)
    cam = scenes.Camera(np.eye(4), 40.0, 44.0, 16.0, 12.0, 32, 24)
    D = torch.tensor(_plane_depth(n, -3.0, cam), dtype=DT)
    nt, ok = losses.depth_normals(D, torch.ones_like(D), cam)
    assert ok[1:-1, 1:-1].all() and not ok[0].any() and not ok[:, -1].any()
    np.testing.assert_allclose(nt[1:-1, 1:-1].numpy(), np.broadcast_to(n, (22, 30, 3)), atol=1e-12)


def test_normal_consistency_definition():
    w = torch.tensor([[0.5, 0.25]], dtype=DT)
    ns = torch.tensor([[[0.0, 0.0, -1.0], [0.6, 0.0, -0.8]]], dtype=DT)
    nt = torch.tensor([[0.0, 0.0, -1.0]], dtype=DT)
    L = losses.normal_consistency(w, ns, nt, torch.tensor([True]))
    assert abs(L.item() - 0.25 * (1 - 0.8)) < 1e-15
    assert losses.normal_consistency(w, ns, nt, torch.tensor([False])).item() == 0.0


def _on_axis(zs, ops, s=0.5):
    """Fronto-parallel splats centred on the optical axis: q = 0, so each has the
    constant planar depth z and the normal (0, 0, -1) over the whole image."""
    n = len(zs)
    return scenes.Scene(np.c_[np.zeros((n, 2)), zs], np.tile([[s, s, 1e-3]], (n, 1)),
                        np.tile([[1.0, 0, 0, 0]], (n, 1)), np.asarray(ops, float),
                        np.zeros((n, 1, 3)), 0)


def test_on_axis_splat_has_no_normal_loss_and_no_distortion():
    cam = scenes.Camera(np.eye(4), 32.0, 32.0, 12.0, 12.0, 24, 24)
    maps, _, _ = losses.render_with_losses(_on_axis([3.0, 3.0], [0.6, 0.5]), cam)
    assert maps["n_ok"].sum() > 300
    assert np.abs(maps["nloss"]).max() < 1e-12
    assert np.abs(maps["dist"]).max() < 1e-12
    ok = maps["n_ok"]
    np.testing.assert_allclose(maps["n_tilde"][ok], np.tile([0.0, 0.0, -1.0], (ok.sum(), 1)), atol=1e-12)


def test_distortion_of_two_on_axis_layers_matches_the_blend_weights():
    # alpha_k = o_k exp(-r^2 / (2 (f^2 s^2 / z_k^2 + lowpass))) at pixel offset r;
    # w1 = alpha1, w2 = alpha2 (1 - alpha1); L_d = 2 w1 w2 (z1 - z2)^2
    f, s, z, o = 32.0, 0.5, (3.0, 4.0), (0.6, 0.7)
    cam = scenes.Camera(np.eye(4), f, f, 12.0, 12.0, 24, 24)
    prm = RenderParams()
    maps, _, _ = losses.render_with_losses(_on_axis(list(z), list(o), s), cam, None, prm)
    jj, ii = np.mgrid[0:24, 0:24] + 0.5
    r2 = ((ii - 12.0) ** 2 + (jj - 12.0) ** 2).reshape(-1)
    a = [ok * np.exp(-0.5 * r2 / (f * f * s * s / zk ** 2 + prm.lowpass)) for zk, ok in zip(z, o)]
    sure = (a[0] > 2 * prm.alpha_min) & (a[1] > 2 * prm.alpha_min)
    ref = 2 * a[0] * a[1] * (1 - a[0]) * (z[0] - z[1]) ** 2
    assert sure.sum() > 200
    np.testing.assert_allclose(maps["dist"][sure], ref[sure], rtol=1e-6)
    np.testing.assert_allclose(maps["alpha"][sure], (1 - (1 - a[0]) * (1 - a[1]))[sure], rtol=1e-6)


def _scene(seed):
    rng = np.random.default_rng(seed)
    n = 6
    means = np.c_[rng.uniform(-0.4, 0.4, (n, 2)), rng.uniform(2.0, 3.0, n)]
    return scenes.Scene(means, rng.uniform(0.15, 0.35, (n, 3)), rng.standard_normal((n, 4)),
                        rng.uniform(0.4, 0.9, n), rng.normal(0, 0.3, (n, 1, 3)), 0)


def _fd_check(sc, grads, L, min_checked):
    checked = 0
    for name in ("means", "scales", "quats", "opacities", "sh"):
        base = np.asarray(getattr(sc, name), np.float64)
        g = grads[name]
        gmax = max(np.abs(grads[k]).max() for k in grads)
        for idx in list(np.ndindex(base.shape))[:40]:
            h = 1e-6 * max(1.0, abs(base[idx]))
            a, b = base.copy(), base.copy()
            a[idx] += h
            b[idx] -= h
            fd = (L(scenes.Scene(**{**sc.__dict__, name: a})) - L(scenes.Scene(**{**sc.__dict__, name: b}))) / (2 * h)
            if abs(g[idx]) > 1e-6 * gmax or abs(fd) > 1e-6 * gmax:
                assert abs(fd - g[idx]) <= 1e-3 * max(abs(g[idx]), 1e-3 * gmax), (name, idx, fd, g[idx])
                checked += 1
    assert checked >= min_checked


CAM_FD = scenes.Camera(np.eye(4), 16.0, 16.0, 10.0, 10.0, 20, 20)
PRM_FD = RenderParams(alpha_min=1e-9, T_min=1e-12)


def _up(which):
    rng = np.random.default_rng(5)
    up = [np.zeros((3, 20, 20)), np.zeros((20, 20)), np.zeros((20, 20)), np.zeros((3, 20, 20)),
          np.zeros((20, 20)), np.zeros((20, 20))]
    up[which] = rng.standard_normal((20, 20))
    return up


def test_normal_loss_gradients_match_central_differences():
    # L_n is differentiated through the weights, the splat normals and the
    # depth-map normals (which depend on the median splats' planar depths)
    sc, up = _scene(3), _up(5)
    maps, pg, _ = losses.render_with_losses(sc, CAM_FD, up, PRM_FD)
    assert maps["margin"].min() > 1e-5 and maps["n_ok"].sum() > 50

    def L(s):
        m, _, _ = losses.render_with_losses(s, CAM_FD, None, PRM_FD)
        return float((m["nloss"] * up[5].reshape(-1)).sum())
    _fd_check(sc, pg, L, 50)


def test_distortion_gradients_match_central_differences_with_frozen_weights():
    # the weights of Eq. 23 are constants: the gradient is the derivative of
    # sum_ij w0_i w0_j (d_i - d_j)^2 with w0 the weights at the base point
    from oracle import binning, composite
    from oracle.render import _leaves, _project
    sc, up = _scene(4), _up(4)
    maps, pg, _ = losses.render_with_losses(sc, CAM_FD, up, PRM_FD)
    pix = np.arange(400)

    def parts(s):
        dec = binning.decide(s.means, s.scales, s.quats, s.opacities, CAM_FD, PRM_FD)
        pre = _project(_leaves(s, False), s, CAM_FD, PRM_FD)
        r = composite.composite(pre, dec, 20, 20, PRM_FD, pix)
        return r["weights"].detach(), r["d_all"].detach(), r["gidx"]

    w0, _, g0 = parts(sc)
    assert (w0 > 0).sum(dim=1).max() >= 3

    def L(s):
        _, d, gi = parts(s)
        assert np.array_equal(gi, g0)
        return float((losses.depth_distortion(w0, d).numpy() * up[4].reshape(-1)).sum())
    _fd_check(sc, pg, L, 40)
