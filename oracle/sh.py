"""Real spherical harmonics up to degree 3, from their definition.

The paper computes a Gaussian's colour c_i "from its spherical harmonics
coefficients and viewing direction" (Sec. 3.1, after Eq. 3) without fixing the
basis.  The oracle uses the standard real basis built from the associated
Legendre functions *with* the Condon-Shortley phase:

    Y_l^0      = K_l^0 P_l^0(cos th)
    Y_l^m (m>0) = sqrt(2) K_l^m P_l^m(cos th) cos(m phi)
    Y_l^m (m<0) = sqrt(2) K_l^|m| P_l^|m|(cos th) sin(|m| phi)
    K_l^m = sqrt((2l+1)/(4 pi) * (l-m)!/(l+m)!)

written in Cartesian form for a unit direction (x, y, z):
sin^m(th) cos(m phi) = Re (x + i y)^m, sin^m(th) sin(m phi) = Im (x + i y)^m and
P_l^m(z) = (-1)^m (1 - z^2)^{m/2} d^m/dz^m P_l(z).  Coefficient index k = l^2 + l + m.

Pinned by tests against scipy.special.sph_harm_y (complex SH) and orthonormality.
"""
from __future__ import annotations

import math

import numpy as np
import torch
from numpy.polynomial import legendre as npleg


def _legendre_derivative_coeffs(l: int, m: int) -> np.ndarray:
    """Power-series coefficients (ascending) of d^m/dz^m P_l(z)."""
    c = np.zeros(l + 1)
    c[l] = 1.0
    d = npleg.legder(c, m) if m > 0 else c
    return npleg.leg2poly(d)


def _norm(l: int, m: int) -> float:
    return math.sqrt((2 * l + 1) / (4 * math.pi) * math.factorial(l - m) / math.factorial(l + m))


def basis(dirs: torch.Tensor, degree: int) -> torch.Tensor:
    """(N, 3) unit directions -> (N, (degree+1)^2) real SH values (differentiable)."""
    x, y, z = dirs[:, 0], dirs[:, 1], dirs[:, 2]
    # Re/Im of (x + i y)^m by repeated complex multiplication
    re = [torch.ones_like(x)]
    im = [torch.zeros_like(x)]
    for m in range(1, degree + 1):
        r, i = re[-1], im[-1]
        re.append(r * x - i * y)
        im.append(r * y + i * x)
    out = []
    for l in range(degree + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            coeffs = _legendre_derivative_coeffs(l, am)
            poly = torch.zeros_like(z)
            for k, ck in enumerate(coeffs):
                if ck != 0.0:
                    poly = poly + ck * z ** k
            cs = (-1.0) ** am  # Condon-Shortley phase
            if m == 0:
                out.append(_norm(l, 0) * poly)
            elif m > 0:
                out.append(math.sqrt(2.0) * _norm(l, am) * cs * poly * re[am])
            else:
                out.append(math.sqrt(2.0) * _norm(l, am) * cs * poly * im[am])
    return torch.stack(out, dim=1)


def colour(sh: torch.Tensor, degree: int, dirs: torch.Tensor) -> torch.Tensor:
    """rgb = max(sum_k c_k Y_k(dir) + 1/2, 0).  ``sh`` is (N, K, 3)."""
    K = (degree + 1) ** 2
    Y = basis(dirs, degree)
    val = (Y[:, :, None] * sh[:, :K, :]).sum(dim=1) + 0.5
    return torch.clamp(val, min=0.0)
