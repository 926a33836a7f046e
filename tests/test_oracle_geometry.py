"""Pins of the oracle's per-Gaussian geometry against closed forms, library
routines and invariants (no GPU).

Each test would fail on a plausible mistake in the oracle: a wrong quaternion
convention, a transposed J or W, a sign error in q or n', a missing z_c/t_c.
"""
import math

import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from oracle import gaussians as G
from oracle.params import RenderParams
from paper_2406_01467_b300 import scenes

DT = torch.float64


def _rand_cov(rng, n, smin=0.01, smax=0.3):
    s = torch.tensor(rng.uniform(smin, smax, (n, 3)), dtype=DT)
    q = torch.tensor(rng.standard_normal((n, 4)), dtype=DT)
    return s, q, G.covariance3d(s, q)


def test_quaternion_matches_scipy():
    rng = np.random.default_rng(0)
    q = rng.standard_normal((50, 4))
    R = G.quat_to_rotmat(torch.tensor(q, dtype=DT)).numpy()
    R_ref = Rotation.from_quat(np.concatenate([q[:, 1:], q[:, :1]], 1)).as_matrix()
    np.testing.assert_allclose(R, R_ref, atol=1e-13)


def test_covariance_is_R_S2_Rt():
    # Eq. 1: eigenvalues of Sigma are the squared scales, eigenvectors the columns of R
    rng = np.random.default_rng(1)
    s, q, Sig = _rand_cov(rng, 20)
    for i in range(20):
        ev = np.sort(np.linalg.eigvalsh(Sig[i].numpy()))
        np.testing.assert_allclose(ev, np.sort(s[i].numpy() ** 2), rtol=1e-12)


def _cam(fx=500.0, fy=450.0, W=640, H=480, view=None):
    return scenes.Camera(np.eye(4) if view is None else view, fx, fy, W / 2, H / 2, W, H)


def test_ray_jacobian_matches_finite_differences():
    # J is the derivative of x -> (fx x/z + cx, fy y/z + cy, |x|)  (Eq. 2, Eq. 8)
    fx, fy = 500.0, 450.0
    x = torch.tensor([[0.3, -0.2, 3.0], [-0.5, 0.4, 2.0], [0.05, 0.1, 5.0]], dtype=DT)
    lims = (-10.0, 10.0, -10.0, 10.0)
    J = G.ray_jacobian(x, fx, fy, lims).numpy()

    def f(p):
        return np.array([fx * p[0] / p[2], fy * p[1] / p[2], np.linalg.norm(p)])

    h = 1e-6
    for i in range(len(x)):
        p = x[i].numpy()
        Jfd = np.stack([(f(p + h * e) - f(p - h * e)) / (2 * h) for e in np.eye(3)], axis=1)
        np.testing.assert_allclose(J[i], Jfd, rtol=1e-7, atol=1e-7)


def test_ray_space_covariance_is_linearised_pushforward():
    # Eq. 2: sample x ~ N(x_c, Sigma_cam) with tiny Sigma; map exactly to ray space;
    # the empirical covariance approaches J Sigma_cam J^T.
    rng = np.random.default_rng(2)
    xc = np.array([0.4, -0.3, 3.0])
    s = torch.tensor([[0.002, 0.001, 0.0015]], dtype=DT)
    q = torch.tensor([[0.9, 0.2, -0.3, 0.1]], dtype=DT)
    Sig = G.covariance3d(s, q)[0].numpy()
    fx, fy = 500.0, 450.0
    J = G.ray_jacobian(torch.tensor(xc[None]), fx, fy, (-10, 10, -10, 10))[0].numpy()
    L = np.linalg.cholesky(Sig)
    pts = xc + rng.standard_normal((400000, 3)) @ L.T
    uvt = np.stack([fx * pts[:, 0] / pts[:, 2], fy * pts[:, 1] / pts[:, 2],
                    np.linalg.norm(pts, axis=1)], 1)
    emp = np.cov(uvt.T)
    ref = J @ Sig @ J.T
    np.testing.assert_allclose(emp, ref, rtol=0.02, atol=0.02 * np.abs(ref).max())


def test_two_routes_for_q_agree():
    # Eq. 13 through the full 3x3 inverse vs the Schur form q = -b^T A^-1
    sc = scenes.tiny_scene(300, seed=3)
    cam = scenes.tiny_camera()
    t = lambda a: torch.tensor(np.asarray(a, np.float64), dtype=DT)
    args = (t(sc.means), t(sc.scales), t(sc.quats), t(sc.opacities), t(sc.sh), 0, cam)
    for lp in (0.0, 0.3):
        prm = RenderParams(lowpass=lp)
        a = G.project(*args, prm, route="schur")
        b = G.project(*args, prm, route="full")
        np.testing.assert_allclose(a["q"].numpy(), b["q"].numpy(), rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(a["n"].numpy(), b["n"].numpy(), rtol=1e-9, atol=1e-12)


def test_phat_times_centre_is_zc():
    # Sec. 3.2 / App. A: p_hat (0, 0, t_c)^T = z_c, i.e. the third entry of q_hat is 1
    rng = np.random.default_rng(4)
    s, q, Sig = _rand_cov(rng, 30)
    xc = torch.tensor(np.c_[rng.uniform(-1, 1, (30, 2)), rng.uniform(2, 5, 30)], dtype=DT)
    J = G.ray_jacobian(xc, 400.0, 400.0, (-10, 10, -10, 10))
    Sray = J @ Sig @ J.transpose(1, 2)
    qhat = G.plane_q_full(Sray)
    z, t = xc[:, 2], xc.norm(dim=1)
    phat = (z / t)[:, None] * qhat
    np.testing.assert_allclose((phat[:, 2] * t).numpy(), z.numpy(), rtol=1e-12)


def test_on_axis_depth_is_conditional_mean_plane():
    # A Gaussian on the optical axis: ray space is a scaling, and the planar
    # depth is the regression plane E[z | x, y] = z_c + S_zxy S_xy^-1 dx of the
    # 3D Gaussian (lowpass 0), with dx the pixel offset back-projected at z_c.
    rng = np.random.default_rng(5)
    f, W, H = 300.0, 200, 200
    cam = _cam(f, f, W, H)
    for trial in range(5):
        zc = rng.uniform(2, 6)
        s = rng.uniform(0.05, 0.4, 3)
        q = rng.standard_normal(4)
        means = torch.tensor([[0.0, 0.0, zc]], dtype=DT)
        out = G.project(means, torch.tensor(np.array([s]), dtype=DT), torch.tensor(np.array([q]), dtype=DT),
                        torch.tensor([0.5], dtype=DT), torch.zeros((1, 1, 3), dtype=DT), 0, cam,
                        RenderParams(lowpass=0.0))
        Sig = G.covariance3d(torch.tensor(np.array([s]), dtype=DT),
                            torch.tensor(np.array([q]), dtype=DT))[0].numpy()
        beta = np.linalg.solve(Sig[:2, :2], Sig[:2, 2])  # S_xy^-1 S_xy,z
        for du, dv in [(3.0, -2.0), (-7.5, 1.25), (0.0, 4.0)]:
            # pixel offset (u - u_c) = -du back-projects to dx = -du * z / f
            dx = np.array([-du * zc / f, -dv * zc / f])
            d_ref = zc + beta @ dx
            d = G.planar_depth(out["z"], out["p"], torch.tensor(du, dtype=DT),
                               torch.tensor(dv, dtype=DT))
            assert abs(d.item() - d_ref) < 1e-12 * zc
        n_ref = np.r_[beta, -1.0]
        n_ref /= np.linalg.norm(n_ref)
        np.testing.assert_allclose(out["n"][0].numpy(), n_ref, atol=1e-12)


def test_normal_is_tangent_plane_of_exact_intersection_surface():
    # Without dilation and clamping, n = J^T n' is parallel to Sigma_cam^-1 x_c,
    # the normal at x_c of the exact camera-space locus {x : x^T Sigma^-1 (x - x_c) = 0}
    # of Eq. 7's maxima; it points toward the camera (n . x_c < 0).
    rng = np.random.default_rng(6)
    V = scenes.look_at((0.3, -0.5, -4.0), (0.1, 0.2, 0.0))
    cam = _cam(600.0, 600.0, 800, 600, V)
    N = 40
    means = torch.tensor(rng.uniform(-0.8, 0.8, (N, 3)), dtype=DT)
    s = torch.tensor(rng.uniform(0.02, 0.3, (N, 3)), dtype=DT)
    q = torch.tensor(rng.standard_normal((N, 4)), dtype=DT)
    out = G.project(means, s, q, torch.full((N,), 0.5, dtype=DT), torch.zeros((N, 1, 3), dtype=DT),
                    0, cam, RenderParams(lowpass=0.0, clamp_margin=10.0))
    Vt = torch.tensor(np.asarray(V, np.float32).astype(np.float64))
    Wm = Vt[:3, :3]
    Sc = Wm @ G.covariance3d(s, q) @ Wm.T
    ref = -torch.linalg.solve(Sc, out["xc"].unsqueeze(-1)).squeeze(-1)
    ref = ref / ref.norm(dim=1, keepdim=True)
    np.testing.assert_allclose(out["n"].numpy(), ref.numpy(), atol=1e-10)
    assert ((out["n"] * out["xc"]).sum(1) < 0).all()


def _eq7_sweep(xc, s, qv, cam, f, rng):
    st, qt = torch.tensor(np.array([s]), dtype=DT), torch.tensor(np.array([qv]), dtype=DT)
    out = G.project(torch.tensor(np.array([xc]), dtype=DT), st, qt, torch.tensor([0.5], dtype=DT),
                    torch.zeros((1, 1, 3), dtype=DT), 0, cam,
                    RenderParams(lowpass=0.0, clamp_margin=10.0))
    Sig = G.covariance3d(st, qt)[0]
    uc, vc = out["u"].item(), out["v"].item()
    z, t = out["z"].item(), out["t"].item()
    dirv = rng.standard_normal(2)
    dirv /= np.linalg.norm(dirv)
    err_t, err_d = [], []
    for r in (4.0, 2.0, 1.0, 0.5):
        u, v = uc - r * dirv[0], vc - r * dirv[1]
        ray = np.array([(u - cam.cx) / f, (v - cam.cy) / f, 1.0])
        ray /= np.linalg.norm(ray)
        d_exact = G.exact_ray_depth(torch.tensor(xc, dtype=DT), Sig,
                                    torch.tensor(ray[None], dtype=DT)).item()
        t_exact = d_exact / ray[2]
        d_plane = G.planar_depth(out["z"], out["p"], torch.tensor(uc - u, dtype=DT),
                                 torch.tensor(vc - v, dtype=DT)).item()
        t_plane = d_plane * t / z            # Eq. 14-15: d = (z_c/t_c) t*
        err_t.append(abs(t_plane - t_exact))
        err_d.append(abs(d_plane - d_exact))
    ray0 = torch.tensor(xc / np.linalg.norm(xc))[None]
    d0 = G.exact_ray_depth(torch.tensor(xc, dtype=DT), Sig, ray0).item()
    return err_t, err_d, d0


def test_ray_space_distance_matches_eq7_to_first_order():
    # Eq. 7 (exact maximum along each camera ray) vs the ray-space maximum of
    # Eq. 12-13: the distances t* agree at the centre pixel and to first order
    # around it (error O(|Delta|^2)).  The depth d = cos(theta_c) t* uses the
    # centre's angle (Eq. 14-15), so off the optical axis the *depth* differs at
    # first order while the *distance* does not.
    rng = np.random.default_rng(7)
    f = 500.0
    cam = _cam(f, f, 640, 480)
    for trial in range(4):
        xc = np.array([rng.uniform(-0.6, 0.6), rng.uniform(-0.4, 0.4), rng.uniform(2.5, 4.0)])
        err_t, err_d, d0 = _eq7_sweep(xc, rng.uniform(0.05, 0.3, 3), rng.standard_normal(4),
                                      cam, f, rng)
        assert abs(d0 - xc[2]) < 1e-12
        for i in range(3):
            assert 3.0 < err_t[i] / err_t[i + 1] < 5.5, err_t


def test_on_axis_depth_matches_eq7_to_first_order():
    # On the optical axis cos(theta) is stationary, so the depth itself agrees
    # with Eq. 7 to first order.
    rng = np.random.default_rng(17)
    f = 500.0
    cam = _cam(f, f, 640, 480)
    for trial in range(3):
        xc = np.array([0.0, 0.0, rng.uniform(2.5, 4.0)])
        err_t, err_d, d0 = _eq7_sweep(xc, rng.uniform(0.05, 0.3, 3), rng.standard_normal(4),
                                      cam, f, rng)
        for i in range(3):
            assert 3.0 < err_d[i] / err_d[i + 1] < 5.5, err_d


def test_flattened_splat_normal_is_plane_normal():
    # A splat flattened along its third axis (scale eps): n -> -+ R e3 with error
    # O(eps^2 / s^2), s the in-plane scale (Sec. 3.3).  Orientations are kept away
    # from grazing so the asymptotic regime starts early.
    rng = np.random.default_rng(8)
    cam = _cam(500.0, 500.0, 640, 480)
    xc = torch.tensor([[0.2, -0.1, 3.0]], dtype=DT)
    xhat = xc[0].numpy() / np.linalg.norm(xc[0].numpy())
    done = 0
    while done < 4:
        qv = torch.tensor(np.array([rng.standard_normal(4)]), dtype=DT)
        R = G.quat_to_rotmat(qv)[0].numpy()
        e3 = R[:, 2]
        if abs(e3 @ xhat) < 0.4:
            continue
        e3 = -e3 if e3 @ xhat > 0 else e3   # oriented toward the camera
        errs = []
        for eps in (4e-3, 2e-3, 1e-3):
            s = torch.tensor([[0.2, 0.15, eps]], dtype=DT)
            out = G.project(xc, s, qv, torch.tensor([0.5], dtype=DT),
                            torch.zeros((1, 1, 3), dtype=DT), 0, cam,
                            RenderParams(lowpass=0.0, clamp_margin=10.0))
            errs.append(np.linalg.norm(out["n"][0].numpy() - e3))
        assert errs[-1] < 1e-3
        for i in range(2):
            assert 3.5 < errs[i] / errs[i + 1] < 4.5, errs
        done += 1


def test_fronto_parallel_flat_splat_on_axis():
    cam = _cam(400.0, 400.0, 320, 240)
    s = torch.tensor([[0.3, 0.2, 1e-4]], dtype=DT)
    qv = torch.tensor([[1.0, 0.0, 0.0, 0.0]], dtype=DT)
    out = G.project(torch.tensor([[0.0, 0.0, 2.5]], dtype=DT), s, qv, torch.tensor([0.5], dtype=DT),
                    torch.zeros((1, 1, 3), dtype=DT), 0, cam, RenderParams(lowpass=0.3))
    np.testing.assert_allclose(out["p"][0].numpy(), [0.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(out["n"][0].numpy(), [0.0, 0.0, -1.0], atol=1e-15)


def test_depth_and_normal_invariant_to_pixel_units():
    # Rescaling the image plane (f -> k f) rescales Delta by k and p by 1/k:
    # the depth along a fixed ray and the camera-space normal do not change.
    rng = np.random.default_rng(9)
    xc = torch.tensor([[0.3, -0.2, 3.0]], dtype=DT)
    s = torch.tensor([rng.uniform(0.05, 0.3, 3)], dtype=DT)
    qv = torch.tensor([rng.standard_normal(4)], dtype=DT)
    res = []
    for k in (1.0, 3.0):
        cam = _cam(300.0 * k, 300.0 * k, int(640 * k), int(480 * k))
        out = G.project(xc, s, qv, torch.tensor([0.5], dtype=DT), torch.zeros((1, 1, 3), dtype=DT),
                        0, cam, RenderParams(lowpass=0.0, clamp_margin=10.0))
        ray = np.array([0.05, -0.03])  # normalised image coordinates of a fixed ray
        u = ray[0] * 300.0 * k + cam.cx
        v = ray[1] * 300.0 * k + cam.cy
        d = G.planar_depth(out["z"], out["p"], out["u"] - u, out["v"] - v).item()
        res.append((d, out["n"][0].numpy()))
    assert abs(res[0][0] - res[1][0]) < 1e-12
    np.testing.assert_allclose(res[0][1], res[1][1], atol=1e-12)
