"""Pins of the oracle's SH colour and FP32 binning (no GPU)."""
import numpy as np
import pytest
import torch
from scipy.special import sph_harm_y

from oracle import binning, gaussians as G, sh as SH
from oracle.params import RenderParams
from paper_2406_01467_b300 import scenes

DT = torch.float64


def _real_sh_scipy(l, m, theta, phi):
    """Real SH from scipy's complex ones (which carry the Condon-Shortley phase)."""
    if m == 0:
        return sph_harm_y(l, 0, theta, phi).real
    Y = sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return np.sqrt(2.0) * Y.real
    return np.sqrt(2.0) * Y.imag


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(0)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    theta = np.arccos(d[:, 2])
    phi = np.arctan2(d[:, 1], d[:, 0])
    Y = SH.basis(torch.tensor(d, dtype=DT), 3).numpy()
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, k], _real_sh_scipy(l, m, theta, phi), atol=1e-12)
            k += 1


def test_sh_basis_is_orthonormal():
    # Gauss-Legendre in cos(theta) x uniform phi integrates degree <= 6 products exactly
    x, w = np.polynomial.legendre.leggauss(8)
    phi = np.arange(16) * 2 * np.pi / 16
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    d = np.stack([st * np.cos(ph), st * np.sin(ph), ct], -1).reshape(-1, 3)
    wt = (w[:, None] * np.full_like(ph, 2 * np.pi / 16)).reshape(-1)
    Y = SH.basis(torch.tensor(d, dtype=DT), 3).numpy()
    gram = (Y * wt[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(16), atol=1e-12)


def test_sh_colour_dc_and_clamp():
    # degree 0: rgb = max(Y00 c + 1/2, 0), independent of direction
    c = torch.tensor([[[1.0, -3.0, 0.0]]], dtype=DT)
    d = torch.tensor([[0.0, 0.6, 0.8]], dtype=DT)
    rgb = SH.colour(c, 0, d).numpy()[0]
    y00 = 0.5 / np.sqrt(np.pi)
    np.testing.assert_allclose(rgb, [y00 + 0.5, max(0.0, -3 * y00 + 0.5), 0.5], atol=1e-15)


def _fp64_ref(scene, cam, params):
    t = lambda a: torch.tensor(np.asarray(a, np.float64), dtype=DT)
    return G.project(t(scene.means), t(scene.scales), t(scene.quats), t(scene.opacities),
                     t(scene.sh), scene.sh_degree, cam, params)


@pytest.mark.parametrize("which", ["tiny", "object_small"])
def test_fp32_decisions_track_fp64_projection(which):
    # The FP32 chain (binning) must compute the same u, v and 2x2 covariance
    # diagonal as the FP64 derivation (Eq. 2), up to FP32 rounding.
    if which == "tiny":
        sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    else:
        sc, cam = scenes.object_scene(5000, seed=11), scenes.object_camera()
    prm = RenderParams()
    dec = binning.decide(sc.means, sc.scales, sc.quats, sc.opacities, cam, prm)
    ref = _fp64_ref(sc, cam, prm)
    v = dec["valid"]
    assert v.sum() > 100
    np.testing.assert_allclose(dec["u"][v], ref["u"].numpy()[v], rtol=0, atol=2e-4)
    np.testing.assert_allclose(dec["v"][v], ref["v"].numpy()[v], rtol=0, atol=2e-4)
    np.testing.assert_allclose(dec["A00"][v], ref["A"][:, 0, 0].numpy()[v], rtol=1e-4)
    np.testing.assert_allclose(dec["A11"][v], ref["A"][:, 1, 1].numpy()[v], rtol=1e-4)
    # culling: z <= near are invalid
    z = ref["z"].numpy()
    assert not (v & (z <= cam.near)).any()


def test_rect_contains_alpha_min_ellipse():
    # For opacity 1 the set alpha >= alpha_min is the ellipse Delta^T conic Delta <= 2 ln(1/alpha_min);
    # every point of it must lie inside the pixel-centre bounds [xlo, xhi] x [ylo, yhi].
    sc, cam = scenes.tiny_scene(500, seed=5), scenes.tiny_camera()
    prm = RenderParams()
    ref = _fp64_ref(sc, cam, prm)
    A = ref["A"].numpy()
    u, v = ref["u"].numpy(), ref["v"].numpy()
    C = 2 * np.log(1.0 / prm.alpha_min)
    th = np.linspace(0, 2 * np.pi, 64, endpoint=False)
    dec = binning.decide(sc.means, sc.scales, sc.quats, sc.opacities, cam, prm)
    for i in range(len(u)):
        L = np.linalg.cholesky(A[i])
        pts = (L @ np.stack([np.cos(th), np.sin(th)])) * np.sqrt(C)
        ex_needed = np.abs(pts[0]).max()
        ey_needed = np.abs(pts[1]).max()
        ex = np.sqrt(np.float32(prm.ext_constant_f32()) * dec["A00"][i])
        ey = np.sqrt(np.float32(prm.ext_constant_f32()) * dec["A11"][i])
        assert ex >= ex_needed * (1 - 1e-5) and ey >= ey_needed * (1 - 1e-5)
        # and the box is tight: the ellipse touches it
        assert ex <= ex_needed * (1 + 2e-3) + 1e-6


def test_tile_lists_brute_force_equals_enumeration():
    sc, cam = scenes.tiny_scene(), scenes.tiny_camera()
    for tw, th in [(16, 16), (8, 8), (32, 8), (16, 4)]:
        prm = RenderParams(tile_w=tw, tile_h=th)
        dec = binning.decide(sc.means, sc.scales, sc.quats, sc.opacities, cam, prm)
        a = binning.tile_lists(dec, cam, prm, brute_force=True)
        b = binning.tile_lists(dec, cam, prm, brute_force=False)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


def test_tile_lists_cover_exactly_the_pixels_of_each_rect():
    # Pixel-level brute force: tile t lists Gaussian g iff some pixel of t lies in g's rect.
    sc, cam = scenes.tiny_scene(300, seed=7), scenes.tiny_camera()
    prm = RenderParams(tile_w=16, tile_h=8)
    dec = binning.decide(sc.means, sc.scales, sc.quats, sc.opacities, cam, prm)
    tile, g, ranges = binning.tile_lists(dec, cam, prm)
    tiles_x, tiles_y = binning.tile_grid(cam, prm)
    expect = set()
    for gi in np.nonzero(dec["valid"])[0]:
        i0, i1, j0, j1 = dec["rect"][gi]
        for j in range(j0, j1 + 1):
            for i in range(i0, i1 + 1):
                expect.add(((j // prm.tile_h) * tiles_x + i // prm.tile_w, gi))
    got = set(zip(tile.tolist(), g.tolist()))
    assert got == expect
    # sorted by (tile, depth bits, id); ranges partition the list
    key = np.stack([tile, dec["zkey"][g].astype(np.int64), g], 1)
    assert (np.diff(key[:, 0]) >= 0).all()
    same = np.diff(key[:, 0]) == 0
    d = np.diff(key[:, 1])
    assert (d[same] >= 0).all()
    assert (np.diff(key[:, 2])[same & (d == 0)] > 0).all()
    assert ranges[:, 1].max() == len(tile)
    for t in range(tiles_x * tiles_y):
        assert (tile[ranges[t, 0]:ranges[t, 1]] == t).all()


def test_behind_camera_and_offscreen_are_culled():
    cam = scenes.tiny_camera()
    m = np.array([[0, 0, -3.0], [0, 0, 0.1], [50, 0, 3.0], [0, 0, 3.0]], np.float32)
    s = np.full((4, 3), 0.05, np.float32)
    q = np.tile(np.array([[1, 0, 0, 0]], np.float32), (4, 1))
    o = np.full(4, 0.5, np.float32)
    dec = binning.decide(m, s, q, o, cam, RenderParams())
    assert dec["valid"].tolist() == [False, False, False, True]
