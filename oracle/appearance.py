"""Decoupled per-view appearance in FP64 (test infrastructure only).

RaDe-GS trains with the decoupled appearance modelling of VastGaussian
(Sec. 4.1.1): a per-view learned code corrects the rendered colours before the
photometric loss, so that exposure and white-balance changes between views are
not baked into the Gaussians.  Reading (the paper gives no architecture): each
training view n owns an embedding e_n in R^E; a two-layer perceptron
    h = relu(W1 e_n + b1),  a = W2 h + b2  (a in R^12)
gives the colour affine M_n = I + [a0 a1 a2; a3 a4 a5; a6 a7 a8], t_n = (a9, a10, a11);
the corrected colour of a pixel is c' = M_n c + t_n and the loss of view n is
the mean over its pixels and channels of |c' - target|.  With W2 = 0 and
b2 = 0 the correction is the identity.  Parameters are trained with Adam
(Kingma and Ba, 2015: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)).

Flat parameter layout (shared with the library's buffers):
    embed [n_emb][E], W1 [H][E], b1 [H], W2 [12][H], b2 [12].
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


def param_count(n_emb: int, E: int, H: int) -> int:
    return n_emb * E + H * E + H + 12 * H + 12


def unpack(flat: torch.Tensor, n_emb: int, E: int, H: int):
    sizes = [n_emb * E, H * E, H, 12 * H, 12]
    parts = torch.split(flat, sizes)
    return (parts[0].view(n_emb, E), parts[1].view(H, E), parts[2], parts[3].view(12, H), parts[4])


def affine(flat: torch.Tensor, n_emb: int, E: int, H: int, idx: int):
    """(M (3,3), t (3,)) of embedding row ``idx``."""
    emb, W1, b1, W2, b2 = unpack(flat, n_emb, E, H)
    h = torch.relu(W1 @ emb[idx] + b1)
    a = W2 @ h + b2
    return torch.eye(3, dtype=flat.dtype) + a[:9].view(3, 3), a[9:]


def loss_and_grads(flat, n_emb, E, H, colors, targets, embed_index):
    """``colors`` / ``targets``: lists of (3, H_v, W_v) arrays; ``embed_index``:
    the embedding row of each view.  Returns (per-view losses, d flat params,
    list of d colour maps, list of corrected maps), all FP64 numpy."""
    p = torch.tensor(np.asarray(flat, np.float64), dtype=DT, requires_grad=True)
    cs = [torch.tensor(np.asarray(c, np.float64), dtype=DT, requires_grad=True) for c in colors]
    losses, corr = [], []
    for c, tgt, k in zip(cs, targets, embed_index):
        M, t = affine(p, n_emb, E, H, int(k))
        cc = torch.einsum("ij,jhw->ihw", M, c) + t[:, None, None]
        corr.append(cc)
        losses.append((cc - torch.tensor(np.asarray(tgt, np.float64), dtype=DT)).abs().mean())
    total = sum(losses)
    grads = torch.autograd.grad(total, [p] + cs)
    return (np.array([l.item() for l in losses]), grads[0].numpy(), [g.numpy() for g in grads[1:]],
            [x.detach().numpy() for x in corr])


def adam(p, g, m, v, step, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (FP64 numpy), returns (p, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def psnr(a, b):
    mse = float(np.mean((np.asarray(a, np.float64) - np.asarray(b, np.float64)) ** 2))
    return 10.0 * np.log10(1.0 / max(mse, 1e-30))
