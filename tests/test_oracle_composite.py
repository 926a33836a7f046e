"""Pins of the oracle's compositing (Eq. 3-4, median depth, normal map) and of
its FP64 gradients (no GPU)."""
import math

import numpy as np
import pytest

import oracle
from oracle import RenderParams
from paper_2406_01467_b300 import scenes


def _scene(means, scales, quats, opac, rgb):
    n = len(means)
    sh = ((np.asarray(rgb, np.float64) - 0.5) / scenes.Y00)[:, None, :]
    return scenes.Scene(np.asarray(means, np.float32), np.asarray(scales, np.float32),
                        np.asarray(quats, np.float32), np.asarray(opac, np.float32),
                        sh.astype(np.float32), 0)


def _cam(W=32, H=32, f=64.0):
    return scenes.Camera(np.eye(4), f, f, W / 2, H / 2, W, H)


def test_single_gaussian_peak_alpha_is_opacity():
    # P1: a Gaussian whose centre projects onto a pixel centre has alpha = o there,
    # colour o * rgb, depth z_c (Delta = 0) and normal o * n (Eq. 3, Eq. 4).
    cam = _cam()
    z = 2.0
    # pixel (10, 20) centre is (10.5, 20.5): x = (u - cx) z / f
    x = (10.5 - 16) * z / 64.0
    y = (20.5 - 16) * z / 64.0
    for o in (0.2, 0.7, 0.95):
        sc = _scene([[x, y, z]], [[0.05, 0.03, 0.02]], [[0.9, 0.1, -0.2, 0.3]], [o],
                    [[0.2, 0.5, 0.9]])
        pix = np.array([20 * 32 + 10])
        r = oracle.render(sc, cam, RenderParams(), pixels=pix)
        rgb = r["pre"]["rgb"][0]
        n = r["pre"]["n"][0]
        o32 = float(np.float32(o))   # inputs are float32
        assert abs(r["alpha"][0] - o32) < 1e-15
        np.testing.assert_allclose(r["color"][0], o32 * rgb, atol=1e-15)
        np.testing.assert_allclose(r["normal"][0], o32 * n, atol=1e-15)
        assert abs(r["depth"][0] - r["pre"]["z"][0]) < 1e-15
    # above alpha_max the alpha is clamped
    sc = _scene([[x, y, z]], [[0.05, 0.03, 0.02]], [[1, 0, 0, 0]], [0.999], [[0.2, 0.5, 0.9]])
    r = oracle.render(sc, cam, RenderParams(), pixels=pix)
    assert abs(r["alpha"][0] - 0.99) < 1e-12


def _stack_at_pixel(opacities, depths, cam, px=(10, 20)):
    """Gaussians centred exactly on one pixel centre at the given depths."""
    means = []
    for z in depths:
        means.append([(px[0] + 0.5 - cam.cx) * z / cam.fx, (px[1] + 0.5 - cam.cy) * z / cam.fy, z])
    n = len(depths)
    rgb = np.linspace(0.1, 0.9, 3 * n).reshape(n, 3)
    return _scene(means, [[0.05, 0.05, 0.05]] * n, [[1, 0, 0, 0]] * n, opacities, rgb), rgb


def test_three_splats_front_to_back_and_median():
    # o = (0.3, 0.4, 0.6) at the pixel centre, listed back to front on purpose.
    # Front to back: T after each = 0.7, 0.42, 0.168; the median (T' <= 0.5) is the second.
    cam = _cam()
    sc, rgb = _stack_at_pixel([0.6, 0.4, 0.3], [3.0, 2.5, 2.0], cam)
    pix = np.array([20 * 32 + 10])
    r = oracle.render(sc, cam, RenderParams(), pixels=pix)
    rgb_f = r["pre"]["rgb"]  # in input order
    f = lambda x: float(np.float32(x))
    w = [f(0.3), (1 - f(0.3)) * f(0.4), (1 - f(0.3)) * (1 - f(0.4)) * f(0.6)]
    order = [2, 1, 0]
    exp_c = sum(wi * rgb_f[g] for wi, g in zip(w, order))
    np.testing.assert_allclose(r["color"][0], exp_c, atol=1e-12)
    assert abs(r["alpha"][0] - (1 - (1 - f(0.3)) * (1 - f(0.4)) * (1 - f(0.6)))) < 1e-12
    assert abs(r["depth"][0] - r["pre"]["z"][1]) < 1e-12


def test_median_falls_back_to_last_contributor():
    cam = _cam()
    sc, _ = _stack_at_pixel([0.2, 0.3], [2.0, 3.0], cam)   # T' = 0.8, 0.56: never <= 0.5
    r = oracle.render(sc, cam, RenderParams(), pixels=np.array([20 * 32 + 10]))
    assert abs(r["depth"][0] - r["pre"]["z"][1]) < 1e-12
    empty = oracle.render(sc, cam, RenderParams(), pixels=np.array([0]))
    assert empty["depth"][0] == 0.0 and empty["alpha"][0] == 0.0


def test_early_termination_drops_the_splat_that_crosses_T_min():
    cam = _cam()
    sc, _ = _stack_at_pixel([0.98, 0.98, 0.98, 0.98], [2.0, 2.2, 2.4, 2.6], cam)
    r = oracle.render(sc, cam, RenderParams(), pixels=np.array([20 * 32 + 10]))
    # T' = 0.02, 4e-4, then 8e-6 < 1e-4 stops: only two splats contribute
    assert r["n_contrib"][0] == 2
    a = float(np.float32(0.98))
    assert abs(r["alpha"][0] - (1 - (1 - a) ** 2)) < 1e-12


def _literal_composite(scene, cam, prm, pre, dec):
    """Plain per-pixel loop written straight from the rules (brute force)."""
    H, W = cam.height, cam.width
    out = np.zeros((H * W, 8))
    valid = np.nonzero(dec["valid"])[0]
    for pix in range(H * W):
        i, j = pix % W, pix // W
        cand = [g for g in valid if dec["rect"][g, 0] <= i <= dec["rect"][g, 1]
                and dec["rect"][g, 2] <= j <= dec["rect"][g, 3]]
        cand.sort(key=lambda g: (int(dec["zkey"][g]), g))
        T, C, N = 1.0, np.zeros(3), np.zeros(3)
        depth, med, last = 0.0, None, None
        for g in cand:
            du = pre["u"][g] - (i + 0.5)
            dv = pre["v"][g] - (j + 0.5)
            a, b, c = pre["conic"][g]
            sig = 0.5 * (a * du * du + c * dv * dv) + b * du * dv
            alpha = min(prm.alpha_max, pre["opacity"][g] * math.exp(-sig))
            if alpha < prm.alpha_min:
                continue
            Tn = T * (1 - alpha)
            if Tn < prm.T_min:
                break
            w = alpha * T
            C += w * pre["rgb"][g]
            N += w * pre["n"][g]
            d = pre["z"][g] + pre["p"][g, 0] * du + pre["p"][g, 1] * dv
            if med is None and Tn <= prm.median_T:
                med = d
            last = d
            T = Tn
        if med is None and last is not None:
            med = last
        out[pix] = [*C, 1 - T, med if med is not None else 0.0, *N]
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_vectorised_composite_equals_literal_loop(seed):
    sc = scenes.tiny_scene(60, seed=20 + seed)
    cam = scenes.Camera(np.eye(4), 24.0, 24.0, 12.0, 10.0, 24, 20)
    prm = RenderParams(alpha_min=1.0 / 255 if seed == 0 else 0.02, T_min=1e-4 if seed == 0 else 0.05)
    r = oracle.render(sc, cam, prm)
    lit = _literal_composite(sc, cam, prm, r["pre"], r["dec"])
    np.testing.assert_allclose(r["color"], lit[:, 0:3], atol=1e-12)
    np.testing.assert_allclose(r["alpha"], lit[:, 3], atol=1e-12)
    np.testing.assert_allclose(r["depth"], lit[:, 4], atol=1e-12)
    np.testing.assert_allclose(r["normal"], lit[:, 5:8], atol=1e-12)


def test_weights_and_final_transmittance_sum_to_one():
    # P6: sum_i w_i + T_final = 1 (telescoping of Eq. 3), alpha map = 1 - T_final
    from oracle import composite as comp
    import torch
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    prm = RenderParams()
    r = oracle.render(sc, cam, prm, pixels=np.arange(0, 128 * 128, 7))
    pre = {k: torch.tensor(v) for k, v in r["pre"].items()}
    c = comp.composite(pre, r["dec"], 128, 128, prm, r["pixels"])
    tot = c["weights"].sum(1) + c["T_final"]
    np.testing.assert_allclose(tot.numpy(), 1.0, atol=1e-13)
    np.testing.assert_allclose(c["alpha"].numpy(), 1 - c["T_final"].numpy(), atol=1e-15)


def test_outputs_do_not_depend_on_tile_size():
    # The pixel-level support rule makes the maps independent of the tile size.
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    pix = np.arange(0, 128 * 128, 5)
    a = oracle.render(sc, cam, RenderParams(tile_w=16, tile_h=16), pixels=pix)
    b = oracle.render(sc, cam, RenderParams(tile_w=8, tile_h=32), pixels=pix)
    for k in ("color", "alpha", "depth", "normal"):
        np.testing.assert_array_equal(a[k], b[k])


# ---------------------------------------------------------------------------
# Gradients: FP64 autograd vs central finite differences (P9)
# ---------------------------------------------------------------------------
def _fd_scene(seed):
    rng = np.random.default_rng(seed)
    n = 6
    means = np.c_[rng.uniform(-0.5, 0.5, (n, 2)), rng.uniform(2.0, 3.0, n)]
    scales = rng.uniform(0.08, 0.3, (n, 3))
    quats = rng.standard_normal((n, 4))
    opac = rng.uniform(0.3, 0.9, n)
    sh = rng.normal(0, 0.3, (n, 4, 3))
    return scenes.Scene(means, scales, quats, opac, sh, 1)


def _loss(scene, cam, prm, up):
    r = oracle.render(scene, cam, prm)
    dC, dA, dD, dN = up
    H, W = cam.height, cam.width
    return float((r["color"] * dC.reshape(3, -1).T).sum() + (r["alpha"] * dA.reshape(-1)).sum()
                 + (r["depth"] * dD.reshape(-1)).sum() + (r["normal"] * dN.reshape(3, -1).T).sum())


@pytest.mark.parametrize("seed", [0, 1])
def test_oracle_gradient_matches_central_differences(seed):
    sc = _fd_scene(seed)
    cam = scenes.Camera(np.eye(4), 20.0, 20.0, 12.0, 12.0, 24, 24)
    # thresholds far from every value so the loss is smooth around the point
    prm = RenderParams(alpha_min=1e-9, T_min=1e-12, lowpass=0.3)
    up = [u[0].astype(np.float64) for u in scenes.upstream_grads(100 + seed, 24, 24)]
    r = oracle.render(sc, cam, prm)
    assert r["margin"].min() > 1e-5   # no decision flips under a 1e-6 step
    pg, g2, _ = oracle.render_grads(sc, cam, up, prm)
    checked = 0
    for name in ("means", "scales", "quats", "opacities", "sh"):
        base = np.asarray(getattr(sc, name), np.float64)
        g = pg[name]
        gmax = np.abs(g).max()
        for idx in np.ndindex(base.shape):
            h = 1e-6 * max(1.0, abs(base[idx]))
            plus, minus = base.copy(), base.copy()
            plus[idx] += h
            minus[idx] -= h
            s1 = scenes.Scene(**{**sc.__dict__, name: plus})
            s0 = scenes.Scene(**{**sc.__dict__, name: minus})
            fd = (_loss(s1, cam, prm, up) - _loss(s0, cam, prm, up)) / (2 * h)
            if abs(g[idx]) > 1e-6 * gmax or abs(fd) > 1e-6 * gmax:
                assert abs(fd - g[idx]) <= 1e-3 * max(abs(g[idx]), 1e-3 * gmax), (name, idx, fd, g[idx])
                checked += 1
    assert checked > 100
