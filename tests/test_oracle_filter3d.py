"""Pins of the oracle's Mip-Splatting 3D filter (Sec. 4.1.1): covariance and
opacity compensation, the render it produces, the variance from the cameras,
and its gradients."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

import oracle
from oracle import filter3d
from oracle import RenderParams
from paper_2406_01467_b300 import scenes


def test_filtered_covariance_is_sigma_plus_v_identity():
    rng = np.random.default_rng(0)
    n = 50
    s = rng.uniform(0.01, 0.5, (n, 3))
    v = rng.uniform(0.0, 0.05, n)
    R = Rotation.random(n, random_state=1).as_matrix()
    st, _ = filter3d.apply_filter(torch.tensor(s), torch.ones(n, dtype=torch.float64), torch.tensor(v))
    st = st.numpy()
    for k in range(n):
        S = R[k] @ np.diag(s[k] ** 2) @ R[k].T
        St = R[k] @ np.diag(st[k] ** 2) @ R[k].T
        np.testing.assert_allclose(St, S + v[k] * np.eye(3), atol=1e-14)


def test_opacity_compensation_keeps_the_integral():
    # o' sqrt(det(Sigma + v I)) = o sqrt(det Sigma): the 3D integral of o G is unchanged
    rng = np.random.default_rng(1)
    n = 40
    s = rng.uniform(0.01, 0.5, (n, 3))
    v = rng.uniform(0.0, 0.05, n)
    o = rng.uniform(0.1, 1.0, n)
    R = Rotation.random(n, random_state=2).as_matrix()
    _, op = filter3d.apply_filter(torch.tensor(s), torch.tensor(o), torch.tensor(v))
    for k in range(n):
        S = R[k] @ np.diag(s[k] ** 2) @ R[k].T
        lhs = op[k].item() * np.sqrt(np.linalg.det(S + v[k] * np.eye(3)))
        assert abs(lhs - o[k] * np.sqrt(np.linalg.det(S))) <= 1e-12 * lhs


def test_fp32_chain_is_the_fp64_filter_rounded():
    rng = np.random.default_rng(2)
    s = rng.uniform(1e-3, 2.0, (1000, 3)).astype(np.float32)
    o = rng.uniform(0.01, 1.0, 1000).astype(np.float32)
    v = rng.uniform(0.0, 0.1, 1000).astype(np.float32)
    st32, op32 = filter3d.apply_filter_f32(s, o, v)
    st, op = filter3d.apply_filter(torch.tensor(s, dtype=torch.float64), torch.tensor(o, dtype=torch.float64),
                                   torch.tensor(v, dtype=torch.float64))
    np.testing.assert_allclose(st32, st.numpy(), rtol=2e-7)
    np.testing.assert_allclose(op32, op.numpy(), rtol=1e-6)


def _single(s, o, z, v=None):
    sc = scenes.Scene(np.array([[0.0, 0.0, z]]), np.array([[s, s, s]]), np.array([[1.0, 0, 0, 0]]),
                      np.array([o]), np.zeros((1, 1, 3)), 0)
    if v is not None:
        sc.filter_var = np.array([v])
    return sc


def test_zero_filter_is_the_identity():
    sc, cam = scenes.tiny_scene(300, seed=3), scenes.tiny_camera()
    a = oracle.render(sc, cam)
    sc.filter_var = np.zeros(sc.n, np.float32)
    b = oracle.render(sc, cam)
    for k in ("color", "alpha", "depth", "normal"):
        np.testing.assert_array_equal(a[k], b[k])


def test_isotropic_splat_render_is_closed_form():
    # on the axis, isotropic: alpha(r) = o (s^2/(s^2+v))^(3/2) exp(-r^2 / (2 (f^2 (s^2+v)/z^2 + 0.3)))
    f, s, o, z, v = 40.0, 0.1, 0.8, 3.0, 0.004
    cam = scenes.Camera(np.eye(4), f, f, 12.0, 12.0, 24, 24)
    prm = RenderParams()
    r = oracle.render(_single(s, o, z, v), cam, prm)
    jj, ii = np.mgrid[0:24, 0:24] + 0.5
    r2 = ((ii - 12.0) ** 2 + (jj - 12.0) ** 2).reshape(-1)
    op = o * (s * s / (s * s + v)) ** 1.5
    ref = op * np.exp(-0.5 * r2 / (f * f * (s * s + v) / z ** 2 + prm.lowpass))
    sure = ref > 2 * prm.alpha_min
    np.testing.assert_allclose(r["alpha"][sure], ref[sure], rtol=1e-6)
    np.testing.assert_allclose(r["depth"][sure], z, rtol=1e-12)


def test_filter_variance_two_views_and_unseen_fill():
    cams = [scenes.Camera(np.eye(4), 100.0, 100.0, 50.0, 50.0, 100, 100),
            scenes.Camera(np.eye(4), 200.0, 200.0, 50.0, 50.0, 100, 100)]
    means = np.array([[0.0, 0.0, 2.0],      # seen by both: min((2/100)^2, (2/200)^2)
                      [0.0, 0.0, -1.0],     # behind both cameras
                      [1.6, 0.0, 2.0]])     # u = 130 > 115 in view 0, u = 210 > 115 in view 1: unseen
    v, seen = filter3d.filter_variance(means, cams)
    assert list(seen) == [True, False, False]
    assert abs(v[0] - 0.2 * (2.0 / 200.0) ** 2) < 1e-18
    assert v[1] == v[0] and v[2] == v[0]
    # the 15 % margin is inclusive: u = -15 (x = -0.65 at z = 2, f = 100) counts as seen
    v2, seen2 = filter3d.filter_variance(np.array([[-1.3, 0.0, 4.0]]), cams[:1])
    assert seen2[0] and abs(v2[0] - 0.2 * (4.0 / 100.0) ** 2) < 1e-18


def test_filter_variance_matches_a_literal_loop():
    rng = np.random.default_rng(4)
    means = np.r_[rng.uniform(-3, 3, (300, 3)), np.c_[rng.uniform(-1, 1, 20), rng.uniform(25, 40, 20),
                                                       rng.uniform(-1, 1, 20)]]   # overhead: seen by no view
    cams = scenes.fusion_cameras(5, seed=1, radius=6.0, width=64, height=48)
    v, seen = filter3d.filter_variance(means, cams)
    ref = []
    for m in means:
        best = None
        for c in cams:
            x = c.viewmat[:3, :3] @ m + c.viewmat[:3, 3]
            if x[2] <= c.near:
                continue
            u, w = c.fx * x[0] / x[2] + c.cx, c.fy * x[1] / x[2] + c.cy
            if -0.15 * c.width <= u <= 1.15 * c.width and -0.15 * c.height <= w <= 1.15 * c.height:
                r = 0.2 * (x[2] / c.fx) ** 2
                best = r if best is None else min(best, r)
        ref.append(best)
    got_seen = [b is not None for b in ref]
    assert list(seen) == got_seen and 0 < sum(got_seen) < len(ref)
    fill = max(b for b in ref if b is not None)
    np.testing.assert_allclose(v, [fill if b is None else b for b in ref], rtol=1e-12)


def test_filtered_gradients_match_central_differences():
    rng = np.random.default_rng(5)
    n = 6
    sc = scenes.Scene(np.c_[rng.uniform(-0.5, 0.5, (n, 2)), rng.uniform(2.0, 3.0, n)],
                      rng.uniform(0.05, 0.25, (n, 3)), rng.standard_normal((n, 4)), rng.uniform(0.3, 0.9, n),
                      rng.normal(0, 0.3, (n, 4, 3)), 1)
    sc.filter_var = rng.uniform(0.001, 0.01, n)
    cam = scenes.Camera(np.eye(4), 20.0, 20.0, 12.0, 12.0, 24, 24)
    prm = RenderParams(alpha_min=1e-9, T_min=1e-12)
    up = [u[0].astype(np.float64) for u in scenes.upstream_grads(7, 24, 24)]
    assert oracle.render(sc, cam, prm)["margin"].min() > 1e-5
    pg, _, _ = oracle.render_grads(sc, cam, up, prm)

    def L(s):
        r = oracle.render(s, cam, prm)
        dC, dA, dD, dN = up
        return float((r["color"] * dC.reshape(3, -1).T).sum() + (r["alpha"] * dA.reshape(-1)).sum()
                     + (r["depth"] * dD.reshape(-1)).sum() + (r["normal"] * dN.reshape(3, -1).T).sum())
    checked = 0
    for name in ("scales", "opacities", "means"):
        base = np.asarray(getattr(sc, name), np.float64)
        g = pg[name]
        gmax = np.abs(g).max()
        for idx in np.ndindex(base.shape):
            h = 1e-6 * max(1.0, abs(base[idx]))
            a, b = base.copy(), base.copy()
            a[idx] += h
            b[idx] -= h
            fd = (L(scenes.Scene(**{**sc.__dict__, name: a})) - L(scenes.Scene(**{**sc.__dict__, name: b}))) / (2 * h)
            if abs(g[idx]) > 1e-6 * gmax or abs(fd) > 1e-6 * gmax:
                assert abs(fd - g[idx]) <= 1e-3 * max(abs(g[idx]), 1e-3 * gmax), (name, idx, fd, g[idx])
                checked += 1
    assert checked > 30
