"""Seeded synthetic scenes and cameras.

This module only draws inputs: Gaussian parameter sets and pinhole cameras.  It
holds none of the rasterizer's arithmetic, so the CUDA path, the FP64 oracle,
the tests and the benchmark can all be fed the same arrays.

Conventions shared by every consumer of these arrays:

* camera frame is OpenCV style (+x right, +y down, +z forward);
* ``viewmat`` is the 4x4 row-major world->camera matrix [R | t];
* a pixel (i, j) is sampled at its centre (i + 0.5, j + 0.5), u = fx*x/z + cx;
* quaternions are (w, x, y, z), unnormalised;
* scales are already activated (> 0), opacities are in (0, 1);
* SH coefficients are stored [N][(deg+1)^2][3], RGB innermost.

All draws are FP64 from ``numpy.random.Generator(PCG64(seed))`` in the order
written in each function, then cast to float32.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np
from scipy.spatial.transform import Rotation

Y00 = 0.28209479177387814  # 1 / (2 sqrt(pi)): the constant SH band, used only to encode DC colours


@dataclass
class Camera:
    viewmat: np.ndarray  # (4, 4) float64, world -> camera
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2

    @property
    def campos(self) -> np.ndarray:
        R = self.viewmat[:3, :3]
        t = self.viewmat[:3, 3]
        return -R.T @ t


@dataclass
class Scene:
    means: np.ndarray      # (N, 3) float32
    scales: np.ndarray     # (N, 3) float32, > 0
    quats: np.ndarray      # (N, 4) float32, (w, x, y, z)
    opacities: np.ndarray  # (N,)   float32, in (0, 1)
    sh: np.ndarray         # (N, K, 3) float32, K = (deg+1)^2
    sh_degree: int
    name: str = ""
    meta: dict = field(default_factory=dict)
    filter_var: Optional[np.ndarray] = None   # (N,) float32 3D-filter variances, or None

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        fv = None if self.filter_var is None else self.filter_var[idx]
        return Scene(self.means[idx], self.scales[idx], self.quats[idx], self.opacities[idx],
                     self.sh[idx], self.sh_degree, self.name + "[subset]", dict(self.meta), fv)


def look_at(eye, target, down=(0.0, 1.0, 0.0)) -> np.ndarray:
    """World->camera [R|t] for an OpenCV camera at ``eye`` looking at ``target``.

    ``down`` is the world direction that should appear downward in the image."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    d = np.asarray(down, np.float64)
    y = d - (d @ z) * z
    y /= np.linalg.norm(y)
    x = np.cross(y, z)
    V = np.eye(4)
    V[0, :3], V[1, :3], V[2, :3] = x, y, z
    V[:3, 3] = -V[:3, :3] @ eye
    return V


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _random_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _quats_from_normals(rng, normals):
    """Quaternions (w,x,y,z) of frames whose local z axis is ``normals``, with a random spin."""
    n = normals / np.linalg.norm(normals, axis=1, keepdims=True)
    spin = rng.uniform(0.0, 2.0 * np.pi, len(n))
    helper = np.where(np.abs(n[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    e1 = np.cross(helper, n)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(n, e1)
    c, s = np.cos(spin)[:, None], np.sin(spin)[:, None]
    a1 = c * e1 + s * e2
    a2 = np.cross(n, a1)
    R = np.stack([a1, a2, n], axis=2)  # columns
    xyzw = Rotation.from_matrix(R).as_quat()
    return np.concatenate([xyzw[:, 3:], xyzw[:, :3]], axis=1)


def _finish(means, log_scales, quats, opac_logits, sh, deg, name, meta=None) -> Scene:
    return Scene(
        means=np.ascontiguousarray(means, np.float32),
        scales=np.ascontiguousarray(np.exp(log_scales), np.float32),
        quats=np.ascontiguousarray(quats, np.float32),
        opacities=np.ascontiguousarray(_sigmoid(opac_logits), np.float32),
        sh=np.ascontiguousarray(sh, np.float32),
        sh_degree=deg, name=name, meta=meta or {})


# ----------------------------------------------------------------------------
# Tiny plain scene: 2,000 Gaussians in front of a 128x128 camera.
# ----------------------------------------------------------------------------
def tiny_scene(n=2000, seed=0) -> Scene:
    """means x,y ~ U[-1,1], z ~ U[2,4]; log-scales N(-3,0.5); random unit quats;
    opacity sigmoid(N(0,1)); SH degree 0 with RGB ~ U(0,1) (stored as (rgb-0.5)/Y00).
    Draw order: xy, z, log-scales, quats, opacity logits, rgb."""
    rng = np.random.Generator(np.random.PCG64(seed))
    xy = rng.uniform(-1.0, 1.0, (n, 2))
    z = rng.uniform(2.0, 4.0, (n, 1))
    ls = rng.normal(-3.0, 0.5, (n, 3))
    q = _random_quats(rng, n)
    ol = rng.normal(0.0, 1.0, n)
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    sh = ((rgb - 0.5) / Y00)[:, None, :]
    return _finish(np.concatenate([xy, z], 1), ls, q, ol, sh, 0, "tiny")


def tiny_camera() -> Camera:
    return Camera(np.eye(4), 128.0, 128.0, 64.0, 64.0, 128, 128)


# ----------------------------------------------------------------------------
# Object-scale scene: noisy sphere-plus-plane shell.
# ----------------------------------------------------------------------------
def _object_points(rng, n):
    n_s = int(round(0.6 * n))
    n_p = n - n_s
    d = rng.standard_normal((n_s, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    sph_pts, sph_nrm = d.copy(), d
    pxz = rng.uniform(-2.0, 2.0, (n_p, 2))
    pl_pts = np.stack([pxz[:, 0], np.ones(n_p), pxz[:, 1]], 1)
    pl_nrm = np.tile([[0.0, -1.0, 0.0]], (n_p, 1))
    pts = np.concatenate([sph_pts, pl_pts])
    nrm = np.concatenate([sph_nrm, pl_nrm])
    pts = pts + nrm * rng.normal(0.0, 0.005, (n, 1))
    return pts, nrm


def object_scene(n=200_000, seed=1, sh_degree=3) -> Scene:
    """60% of the points on the unit sphere, 40% on the plane y=+1 over [-2,2]^2,
    displaced along the normal by N(0, 0.005); log-scales N(-5,0.4) with the normal
    axis scaled x0.1; SH coefficients N(0,0.2); opacity sigmoid(N(1,1)).
    Draw order: sphere dirs, plane xz, noise, log-scales, spins, SH, opacity logits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    pts, nrm = _object_points(rng, n)
    ls = rng.normal(-5.0, 0.4, (n, 3))
    ls[:, 2] += np.log(0.1)
    q = _quats_from_normals(rng, nrm)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.2, (n, K, 3))
    ol = rng.normal(1.0, 1.0, n)
    return _finish(pts, ls, q, ol, sh, sh_degree, "object")


def object_camera(width=800, height=600, f=1100.0) -> Camera:
    return Camera(look_at((0.0, -0.8, -4.0), (0.0, 0.0, 0.0)), f, f, width / 2.0, height / 2.0,
                  width, height)


# ----------------------------------------------------------------------------
# Unbounded scene: planes and spheres in a 10 m box plus a far background shell.
# ----------------------------------------------------------------------------
def unbounded_scene(n=3_000_000, seed=2, sh_degree=3, n_planes=16, n_spheres=16) -> Scene:
    """80% of the Gaussians on 16 random squares (side U[1,4]) and 16 spheres
    (radius U[0.3,1.5]) with centres in [-5,5]^3, allotted by area, displaced
    along the normal by N(0, 0.005), log-scales N(-4,0.5) with the normal axis
    x0.1; 20% on a shell of radius U[50,100] with uniform directions, log-scales
    N(-1,0.7) and random quats.  SH N(0,0.2); opacity sigmoid(N(0,1.5)).
    Draw order: plane centres, normals, sides; sphere centres, radii; per-point
    assignment; plane uv; sphere dirs; noise; fg log-scales; fg spins; shell
    dirs, radii, log-scales, quats; SH; opacity logits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_fg = int(round(0.8 * n))
    n_bg = n - n_fg
    pc = rng.uniform(-5.0, 5.0, (n_planes, 3))
    pn = rng.standard_normal((n_planes, 3))
    pn /= np.linalg.norm(pn, axis=1, keepdims=True)
    side = rng.uniform(1.0, 4.0, n_planes)
    sc = rng.uniform(-5.0, 5.0, (n_spheres, 3))
    sr = rng.uniform(0.3, 1.5, n_spheres)
    area = np.concatenate([side ** 2, 4.0 * np.pi * sr ** 2])
    which = rng.choice(n_planes + n_spheres, size=n_fg, p=area / area.sum())
    which.sort()
    is_plane = which < n_planes
    n_pl = int(is_plane.sum())
    n_sp = n_fg - n_pl
    # plane points
    pid = which[:n_pl]
    uv = rng.uniform(-0.5, 0.5, (n_pl, 2)) * side[pid, None]
    helper = np.where(np.abs(pn[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    t1 = np.cross(helper, pn)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(pn, t1)
    pl_pts = pc[pid] + uv[:, :1] * t1[pid] + uv[:, 1:] * t2[pid]
    pl_nrm = pn[pid]
    # sphere points
    sid = which[n_pl:] - n_planes
    d = rng.standard_normal((n_sp, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    sp_pts = sc[sid] + sr[sid, None] * d
    fg_pts = np.concatenate([pl_pts, sp_pts])
    fg_nrm = np.concatenate([pl_nrm, d])
    fg_pts = fg_pts + fg_nrm * rng.normal(0.0, 0.005, (n_fg, 1))
    fg_ls = rng.normal(-4.0, 0.5, (n_fg, 3))
    fg_ls[:, 2] += np.log(0.1)
    fg_q = _quats_from_normals(rng, fg_nrm)
    # background shell
    bd = rng.standard_normal((n_bg, 3))
    bd /= np.linalg.norm(bd, axis=1, keepdims=True)
    br = rng.uniform(50.0, 100.0, (n_bg, 1))
    bg_pts = bd * br
    bg_ls = rng.normal(-1.0, 0.7, (n_bg, 3))
    bg_q = _random_quats(rng, n_bg)
    K = (sh_degree + 1) ** 2
    sh = rng.normal(0.0, 0.2, (n, K, 3))
    ol = rng.normal(0.0, 1.5, n)
    pts = np.concatenate([fg_pts, bg_pts])
    ls = np.concatenate([fg_ls, bg_ls])
    q = np.concatenate([fg_q, bg_q])
    return _finish(pts, ls, q, ol, sh, sh_degree, "unbounded", {"n_fg": n_fg, "n_bg": n_bg})


def unbounded_camera(width=1297, height=840, f=1150.0, eye=(0.0, 0.0, -7.0)) -> Camera:
    return Camera(look_at(eye, (0.0, 0.0, 0.0)), f, f, width / 2.0, height / 2.0, width, height)


def orbit_cameras(n_views=16, seed=3, radius=7.0):
    """Views on a radius-7 orbit (y = 0 plane) at k*360/n degrees with image sizes
    W ~ U{512..1600}, H ~ U{384..1200} drawn independently, f = 1150*W/1297."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ws = rng.integers(512, 1601, n_views)
    Hs = rng.integers(384, 1201, n_views)
    cams = []
    for k in range(n_views):
        a = 2.0 * np.pi * k / n_views
        eye = (radius * np.sin(a), 0.0, -radius * np.cos(a))
        W, H = int(Ws[k]), int(Hs[k])
        f = 1150.0 * W / 1297.0
        cams.append(Camera(look_at(eye, (0.0, 0.0, 0.0)), f, f, W / 2.0, H / 2.0, W, H))
    return cams


def fusion_cameras(n_views=48, seed=6, radius=7.0, width=1297, height=840):
    """Views for fusing depth into a volume: yaw k*360/n on a radius-7 orbit,
    elevation ~ U[-0.3, 0.3] rad, all W x H with f = 1150 W / 1297, looking at
    the origin."""
    rng = np.random.Generator(np.random.PCG64(seed))
    el = rng.uniform(-0.3, 0.3, n_views)
    f = 1150.0 * width / 1297.0
    cams = []
    for k in range(n_views):
        a = 2.0 * np.pi * k / n_views
        eye = (radius * np.cos(el[k]) * np.sin(a), radius * np.sin(el[k]), -radius * np.cos(el[k]) * np.cos(a))
        cams.append(Camera(look_at(eye, (0.0, 0.0, 0.0)), f, f, width / 2.0, height / 2.0, width, height))
    return cams


def upstream_grads(rng_seed, height, width, n_views=1):
    """Seeded dL/d(colour, alpha, depth, normal) maps, N(0,1) each, FP32."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    sh = (n_views, height, width)
    return (rng.standard_normal((n_views, 3, height, width)).astype(np.float32),
            rng.standard_normal(sh).astype(np.float32),
            rng.standard_normal(sh).astype(np.float32),
            rng.standard_normal((n_views, 3, height, width)).astype(np.float32))


def loss_upstream(rng_seed, height, width, n_views=1):
    """Seeded dL/d(depth distortion, normal consistency) maps, N(0,1) each, FP32."""
    rng = np.random.Generator(np.random.PCG64(rng_seed))
    sh = (n_views, height, width)
    return rng.standard_normal(sh).astype(np.float32), rng.standard_normal(sh).astype(np.float32)


def to_bf16_rounded(a: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even float32 -> bfloat16, returned widened back to float32."""
    a = np.ascontiguousarray(a, np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).reshape(a.shape)
