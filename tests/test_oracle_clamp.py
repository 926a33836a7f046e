"""Pins of the oracle's clamp of x/z and y/z inside the Jacobian (no GPU).

The paper keeps the 3D GS defaults (Sec. 4.1.1).  One of them is that the
perspective rows of J (Eq. 2) are evaluated with x/z and y/z clamped to the
image widened by a margin (here 15 % of its size on each side).  That changes
the screen covariance, the conic, the depth plane (Eq. 13-17) and the normal
(Eq. 22) of splats whose centre projects outside the widened image, and only
those.  The tests below fix the reading from outside the oracle's code:

* the limits are the widened image's borders, hand-computed for a camera whose
  principal point is off centre and whose focal lengths differ;
* the clamped rows are the pinhole derivative taken at the point of the same
  depth whose projection is clamped (finite differences of u = fx x/z + cx),
  and the third row (the derivative of |x|) is not clamped;
* beyond a limit the clamped entry does not move with the centre;
* an isotropic splat beyond the right border renders the closed-form alpha,
  depth and normal of the clamped Jacobian, which differ from the unclamped
  ones;
* the FP64 gradients with the clamp engaged match central differences.

A plausible mistake -- margin applied to one side only or scaled by the wrong
image side, cx in place of W - cx, the clamp applied to u instead of x/z, the
third row clamped too -- fails one of them.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import RenderParams
from oracle import gaussians as G
from oracle.params import clamp_limits_f32
from paper_2406_01467_b300 import scenes

DT = torch.float64

# camera of the hand computations: 100 x 80 pixels, fx = 100, fy = 125,
# principal point (30, 50) (off centre), margin 0.15 -> the widened image is
# u in [-15, 115], v in [-12, 92] pixels.
W_, H_, FX, FY, CX, CY, M = 100, 80, 100.0, 125.0, 30.0, 50.0, 0.15
# x/z = (u - cx) / fx at the widened borders
LIMS = ((-15 - 30) / 100.0, (115 - 30) / 100.0, (-12 - 50) / 125.0, (92 - 50) / 125.0)
#      = (-0.45, 0.85, -0.496, 0.336)


def test_clamp_limits_are_the_widened_image_borders():
    got = clamp_limits_f32(W_, H_, FX, FY, CX, CY, M)
    np.testing.assert_allclose(got, LIMS, rtol=1e-7)
    assert np.float32(got[1]) == np.float32(0.85) and np.float32(got[2]) == np.float32(-0.496)
    # a centred camera gives symmetric limits
    sym = clamp_limits_f32(W_, H_, FX, FY, W_ / 2, H_ / 2, M)
    np.testing.assert_allclose(sym, (-0.65, 0.65, -0.416, 0.416), rtol=1e-7)


def _pinhole(p):
    return np.array([FX * p[0] / p[2] + CX, FY * p[1] / p[2] + CY])


def _fd(f, p, h=1e-6):
    return np.stack([(f(p + h * e) - f(p - h * e)) / (2 * h) for e in np.eye(3)], axis=1)


@pytest.mark.parametrize("txy", [(0.3, -0.1), (1.4, 0.0), (-0.9, 0.2), (0.5, 0.7), (-2.0, -1.5),
                                 (0.85 + 1e-3, 0.336 + 1e-3)])
def test_clamped_jacobian_is_pinhole_derivative_at_clamped_point(txy):
    z = 3.0
    x = np.array([txy[0] * z, txy[1] * z, z])
    J = G.ray_jacobian(torch.tensor(x[None], dtype=DT), FX, FY, LIMS)[0].numpy()
    # the point of the same depth whose projection lies on the widened image
    xc = np.array([min(max(txy[0], LIMS[0]), LIMS[1]) * z, min(max(txy[1], LIMS[2]), LIMS[3]) * z, z])
    Juv = _fd(_pinhole, xc)
    np.testing.assert_allclose(J[:2], Juv, rtol=1e-7, atol=1e-7)
    # the third row is the derivative of |x| at the true centre
    Jt = _fd(lambda p: np.array([np.linalg.norm(p)]), x)
    np.testing.assert_allclose(J[2:], Jt, rtol=1e-7, atol=1e-9)
    clamped = not (LIMS[0] <= txy[0] <= LIMS[1] and LIMS[2] <= txy[1] <= LIMS[3])
    if clamped:   # and it differs from the unclamped derivative
        assert np.abs(J[:2] - _fd(_pinhole, x)).max() > 1e-3


def test_clamped_entry_does_not_move_with_the_centre():
    # dJ02/dx = -fx / z^2 inside the widened image, 0 beyond it (and likewise J12 in y)
    z, h = 2.0, 1e-6
    for tx, inside in ((0.2, True), (0.84, True), (0.86, False), (3.0, False), (-0.46, False)):
        def j02(xv):
            return G.ray_jacobian(torch.tensor([[xv, 0.1, z]], dtype=DT), FX, FY, LIMS)[0, 0, 2].item()
        d = (j02(tx * z + h) - j02(tx * z - h)) / (2 * h)
        assert abs(d - (-FX / z ** 2 if inside else 0.0)) < 1e-6, (tx, d)
    for ty, inside in ((0.0, True), (0.33, True), (0.34, False), (-0.5, False)):
        def j12(yv):
            return G.ray_jacobian(torch.tensor([[0.1, yv, z]], dtype=DT), FX, FY, LIMS)[0, 1, 2].item()
        d = (j12(ty * z + h) - j12(ty * z - h)) / (2 * h)
        assert abs(d - (-FY / z ** 2 if inside else 0.0)) < 1e-6, (ty, d)


def _offscreen_sphere(tx=1.05, z=4.0, s=0.9, o=0.8):
    means = np.array([[tx * z, 0.0, z]], np.float32)
    sh = np.full((1, 1, 3), (0.7 - 0.5) / scenes.Y00, np.float32)
    return scenes.Scene(means, np.full((1, 3), s, np.float32), np.array([[1, 0, 0, 0]], np.float32),
                        np.array([o], np.float32), sh, 0)


def _closed_form(tx, z, s, o, L, lp, px):
    """Alpha, depth and normal of an isotropic splat centred at (tx z, 0, z) at
    pixel centres px (u, v), identity camera pose, with x/z clamped to L inside J.
    J rows: (fx/z, 0, -fx L/z), (0, fy/z, 0), (tx, 0, 1) z/t; Sigma = s^2 I."""
    t = z * math.sqrt(tx * tx + 1)
    A00 = s * s * FX * FX * (1 + L * L) / z ** 2 + lp
    A11 = s * s * FY * FY / z ** 2 + lp
    du = FX * tx + CX - px[:, 0]
    dv = 0.0 + CY - px[:, 1]
    alpha = o * np.exp(-0.5 * (du * du / A00 + dv * dv / A11))
    # b = Sigma'[0:2, 2] = s^2 (j1 . j3, j2 . j3); q = -b A^-1; p = (z/t) q (Eq. 13-15)
    b0 = s * s * (FX / z) * (tx * z - L * z) / t
    q0 = -b0 / A00
    depth = z + (z / t) * q0 * du
    n = np.array([FX / z * -q0 + tx * z / t * -1.0, 0.0, -FX * L / z * -q0 + z / t * -1.0])
    return alpha, depth, n / np.linalg.norm(n)


def test_offscreen_isotropic_splat_renders_the_clamped_closed_form():
    cam = scenes.Camera(np.eye(4), FX, FY, CX, CY, W_, H_)
    tx, z, s, o = 1.05, 4.0, 0.9, 0.8   # u_c = 135: beyond the widened border at 115
    sc = _offscreen_sphere(tx, z, s, o)
    prm = RenderParams()
    cols = np.array([W_ - 1, W_ - 2, W_ - 5, W_ - 12])
    rows = np.array([CY - 0.5 - 3, CY - 0.5, CY - 0.5 + 7]).astype(int)
    pix = (rows[:, None] * W_ + cols[None, :]).reshape(-1)
    px = np.stack([pix % W_ + 0.5, pix // W_ + 0.5], 1)
    r = oracle.render(sc, cam, prm, pixels=pix)
    alpha, depth, n = _closed_form(tx, z, s, o, float(np.float32(LIMS[1])), prm.lowpass, px)
    assert (alpha > prm.alpha_min).all()      # every pixel sees the splat
    np.testing.assert_allclose(r["alpha"], alpha, rtol=1e-6)
    np.testing.assert_allclose(r["color"], np.repeat(alpha[:, None] * 0.7, 3, 1), rtol=1e-6)
    np.testing.assert_allclose(r["depth"], depth, rtol=1e-6)
    np.testing.assert_allclose(r["normal"], alpha[:, None] * n[None], rtol=1e-6, atol=1e-12)
    # without the clamp (L = tx): the depth plane is fronto-parallel and alpha differs
    a_u, d_u, n_u = _closed_form(tx, z, s, o, tx, prm.lowpass, px)
    np.testing.assert_allclose(d_u, z, rtol=1e-12)
    assert np.abs(alpha / a_u - 1).max() > 0.05 and np.abs(depth - z).max() > 1e-2
    r_u = oracle.render(sc, cam, RenderParams(clamp_margin=10.0), pixels=pix)
    np.testing.assert_allclose(r_u["alpha"], a_u, rtol=1e-6)
    np.testing.assert_allclose(r_u["depth"], d_u, rtol=1e-9)


def _clamp_fd_scene(seed):
    """Three splats on screen and three large ones centred beyond different
    borders of the widened image (their J clamps) whose footprints reach it."""
    rng = np.random.default_rng(seed)
    on = np.c_[rng.uniform(-0.3, 0.3, (3, 2)), rng.uniform(2.0, 3.0, 3)]
    z = rng.uniform(2.5, 3.5, 3)
    off = np.stack([[1.25 * z[0], 0.1 * z[0], z[0]], [-0.4 * z[1], -1.5 * z[1], z[1]],
                    [1.1 * z[2], 0.9 * z[2], z[2]]])
    means = np.concatenate([on, off])
    scales = np.concatenate([rng.uniform(0.08, 0.25, (3, 3)), rng.uniform(0.5, 0.9, (3, 3))])
    quats = rng.standard_normal((6, 4))
    opac = rng.uniform(0.3, 0.9, 6)
    sh = rng.normal(0, 0.3, (6, 4, 3))
    return scenes.Scene(means, scales, quats, opac, sh, 1)


def _loss(scene, cam, prm, up):
    r = oracle.render(scene, cam, prm)
    dC, dA, dD, dN = up
    return float((r["color"] * dC.reshape(3, -1).T).sum() + (r["alpha"] * dA.reshape(-1)).sum()
                 + (r["depth"] * dD.reshape(-1)).sum() + (r["normal"] * dN.reshape(3, -1).T).sum())


def test_oracle_gradient_with_clamp_engaged_matches_central_differences():
    sc = _clamp_fd_scene(3)
    cam = scenes.Camera(np.eye(4), 20.0, 20.0, 12.0, 12.0, 24, 24)
    prm = RenderParams(alpha_min=1e-9, T_min=1e-12)
    lims = clamp_limits_f32(24, 24, 20.0, 20.0, 12.0, 12.0, prm.clamp_margin)
    r = oracle.render(sc, cam, prm)
    pre = r["pre"]
    tx = (pre["u"] - 12.0) / 20.0
    ty = (pre["v"] - 12.0) / 20.0
    outside = (tx < lims[0]) | (tx > lims[1]) | (ty < lims[2]) | (ty > lims[3])
    np.testing.assert_array_equal(outside, [False] * 3 + [True] * 3)
    assert r["dec"]["valid"].all() and r["margin"].min() > 1e-5
    up = [u[0].astype(np.float64) for u in scenes.upstream_grads(77, 24, 24)]
    pg, _, _ = oracle.render_grads(sc, cam, up, prm)
    checked = 0
    for name in ("means", "scales", "quats", "opacities"):
        base = np.asarray(getattr(sc, name), np.float64)
        g = pg[name]
        gmax = np.abs(g).max()
        for idx in np.ndindex(base.shape):
            if idx[0] < 3:
                continue   # the on-screen splats are covered by the other FD pins
            h = 1e-6 * max(1.0, abs(base[idx]))
            plus, minus = base.copy(), base.copy()
            plus[idx] += h
            minus[idx] -= h
            fd = (_loss(scenes.Scene(**{**sc.__dict__, name: plus}), cam, prm, up)
                  - _loss(scenes.Scene(**{**sc.__dict__, name: minus}), cam, prm, up)) / (2 * h)
            if abs(g[idx]) > 1e-6 * gmax or abs(fd) > 1e-6 * gmax:
                assert abs(fd - g[idx]) <= 1e-3 * max(abs(g[idx]), 1e-3 * gmax), (name, idx, fd, g[idx])
                checked += 1
    assert checked >= 25
