"""Per-Gaussian quantities in FP64 (torch CPU ops, differentiable by autograd).

Every step follows the paper's derivation in its own order and notation:

* Eq. 1:  Sigma = R S S^T R^T from a unit quaternion and scales.
* Eq. 2:  Sigma' = J W Sigma W^T J^T, the covariance in ray space; the 2D screen
          covariance is its top-left 2x2 block.
* Eq. 8:  ray space u = (u, v, t) with t = |x| the distance to the camera centre,
          so the third row of J is the derivative of |x|, x_c^T / t_c.
* Eq. 13: q_hat = v'^T Sigma'^-1 / (v'^T Sigma'^-1 v'), v' = (0, 0, 1).
* Eq. 15: p_hat = (z_c / t_c) q_hat; p is its first two entries (Eq. 4, 17).
* Eq. 19-21: q = (t_c / z_c) p; ray-space plane normal n' = -(q, 1).
* Eq. 22: camera-space normal n = J^T n', normalised.

Two independent routes give q (and so p and n): the full 3x3 inverse of Eq. 13
and the 2x2 Schur-complement form q = -b^T A^-1 (b = Sigma'[0:2, 2]); the tests
check that they agree.

The screen low-pass (3D GS default) adds ``lowpass`` to the diagonal of the 2x2
block; the same dilated matrix is used for the conic and, in both routes, for
the depth plane (Sigma'_d = Sigma' + diag(lowpass, lowpass, 0)).
"""
from __future__ import annotations

import numpy as np
import torch

from . import sh as shmod
from .params import RenderParams, clamp_limits_f32

DT = torch.float64


def camera_tensors(cam):
    """Camera values as the GPU sees them: rounded to float32, then promoted."""
    f32 = np.float32
    V = torch.tensor(np.asarray(cam.viewmat, f32).astype(np.float64), dtype=DT)
    vals = [float(f32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy)]
    return V, vals


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """(N,4) quaternions (w,x,y,z), normalised here -> (N,3,3) rotation matrices."""
    q = q / q.norm(dim=1, keepdim=True)
    w, x, y, z = q.unbind(1)
    R = torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1),
    ], dim=1)
    return R


def covariance3d(scales: torch.Tensor, quats: torch.Tensor) -> torch.Tensor:
    """Eq. 1: Sigma = R S S^T R^T."""
    R = quat_to_rotmat(quats)
    S = torch.diag_embed(scales)
    RS = R @ S
    return RS @ RS.transpose(1, 2)


def ray_jacobian(xc: torch.Tensor, fx, fy, lims) -> torch.Tensor:
    """Jacobian of x -> (u, v, t) at the centre (Eq. 2's J with Eq. 8's t = |x|).

    Rows 1-2 are the perspective derivative fx/z, -fx x/z^2 (the x/z, y/z inside
    them clamped to ``lims``, a 3D GS default); row 3 is x^T/|x|."""
    x, y, z = xc.unbind(1)
    t = xc.norm(dim=1)
    txc = torch.clamp(x / z, lims[0], lims[1])
    tyc = torch.clamp(y / z, lims[2], lims[3])
    zero = torch.zeros_like(z)
    J = torch.stack([
        torch.stack([fx / z, zero, -fx * txc / z], -1),
        torch.stack([zero, fy / z, -fy * tyc / z], -1),
        torch.stack([x / t, y / t, z / t], -1),
    ], dim=1)
    return J


def plane_q_full(Sd: torch.Tensor) -> torch.Tensor:
    """Eq. 13 with the full 3x3 inverse: q_hat = e3^T Sd^-1 / (e3^T Sd^-1 e3)."""
    Si = torch.linalg.inv(Sd)
    row = Si[:, 2, :]
    return row / row[:, 2:3]


def plane_q_schur(A: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
    """First two entries of q_hat via the Schur complement: q = -b^T A^-1."""
    return -torch.linalg.solve(A, b.unsqueeze(-1)).squeeze(-1)


def camera_normal(J: torch.Tensor, q: torch.Tensor) -> torch.Tensor:
    """Eq. 21-22: n' = -(q, 1), n = J^T n' normalised."""
    nprime = -torch.cat([q, torch.ones_like(q[:, :1])], dim=1)
    n = (J.transpose(1, 2) @ nprime.unsqueeze(-1)).squeeze(-1)
    return n / n.norm(dim=1, keepdim=True)


def project(means, scales, quats, opacities, sh, sh_degree, cam, params: RenderParams,
            route: str = "schur"):
    """All per-Gaussian 2D quantities for one camera.

    Inputs are FP64 torch tensors (leaves may require grad).  Returns a dict of
    (N, ...) tensors: xc, z, t, u, v (pixel coords), J, Sigma_ray (3x3, undilated),
    A (dilated 2x2), det, conic (a, b, c) = A^-1 entries, q, p, n, rgb, opacity.
    ``route`` selects how q is computed ("schur" or "full")."""
    V, (fx, fy, cx, cy) = camera_tensors(cam)
    W = V[:3, :3]
    tw = V[:3, 3]
    lims = clamp_limits_f32(cam.width, cam.height, fx, fy, cx, cy, params.clamp_margin)

    xc = means @ W.T + tw
    z = xc[:, 2]
    t = xc.norm(dim=1)
    u = fx * xc[:, 0] / z + cx
    v = fy * xc[:, 1] / z + cy

    Sigma = covariance3d(scales, quats)
    J = ray_jacobian(xc, fx, fy, lims)
    JW = J @ W
    Sray = JW @ Sigma @ JW.transpose(1, 2)          # Eq. 2
    lp = params.lowpass
    A = Sray[:, :2, :2] + lp * torch.eye(2, dtype=DT)
    det = A[:, 0, 0] * A[:, 1, 1] - A[:, 0, 1] * A[:, 1, 0]
    conic = torch.stack([A[:, 1, 1] / det, -A[:, 0, 1] / det, A[:, 0, 0] / det], dim=1)
    b = Sray[:, :2, 2]
    if route == "schur":
        q = plane_q_schur(A, b)
    else:
        Sd = Sray + torch.diag(torch.tensor([lp, lp, 0.0], dtype=DT))
        q = plane_q_full(Sd)[:, :2]
    p = (z / t).unsqueeze(1) * q                     # Eq. 15, 17
    n = camera_normal(J, q)                          # Eq. 21-22

    campos = -W.T @ tw
    d = means - campos
    dirs = d / d.norm(dim=1, keepdim=True)
    rgb = shmod.colour(sh, sh_degree, dirs)
    return dict(xc=xc, z=z, t=t, u=u, v=v, J=J, Sigma=Sigma, Sigma_ray=Sray, A=A, det=det,
                conic=conic, q=q, p=p, n=n, rgb=rgb, opacity=opacities, dirs=dirs)


def planar_depth(z, p, du, dv):
    """Eq. 4: d = z_c + p (du, dv)^T, du = u_c - u, dv = v_c - v."""
    return z + p[..., 0] * du + p[..., 1] * dv


def exact_ray_depth(xc, Sigma_cam, ray_dirs):
    """Eq. 7 in camera space (camera centre o = 0): the distance t* that maximises
    the Gaussian along each unit ray v, times v_z to give a depth."""
    Si = torch.linalg.inv(Sigma_cam)
    num = torch.einsum("ri,ij,j->r", ray_dirs, Si, xc)
    den = torch.einsum("ri,ij,rj->r", ray_dirs, Si, ray_dirs)
    tstar = num / den
    return tstar * ray_dirs[:, 2]
