"""Decoupled per-view appearance (Sec. 4.1.1, after VastGaussian), trained with
the library's own kernels (gs_appearance_fwd_bwd, gs_adam_step).

Each training view owns an embedding; a two-layer perceptron maps it to a
colour affine c' = (I + A) c + t that is applied to the rendered colour before
the L1 photometric loss.  ``fwd_bwd`` returns the per-view losses and dL/dc,
which is the colour gradient to hand to ``Frame.backward``; ``step`` applies
Adam to the appearance parameters and clears their gradients.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import GsAppearance, check


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Appearance:
    def __init__(self, n_embeddings: int, embed_dim: int = 32, hidden: int = 64, device="cuda", seed: int = 0):
        self.lib = _lib.load()
        n = self.lib.gs_appearance_param_count(n_embeddings, embed_dim, hidden)
        if n == 0:
            check(_lib.GS_ERR_INVALID_ARG, "gs_appearance_param_count")
        self.n_embeddings, self.embed_dim, self.hidden = n_embeddings, embed_dim, hidden
        g = torch.Generator().manual_seed(seed)
        emb = torch.randn(n_embeddings * embed_dim, generator=g) * 0.1
        W1 = torch.randn(hidden * embed_dim, generator=g) / np.sqrt(embed_dim)
        rest = torch.zeros(hidden + 12 * hidden + 12)   # b1, W2, b2: the identity correction
        self.params = torch.cat([emb, W1, rest]).to(device=device, dtype=torch.float32).contiguous()
        assert self.params.numel() == n
        self.grads = torch.zeros_like(self.params)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.device = self.params.device
        self._c = GsAppearance(n_embeddings, embed_dim, hidden, 0, _ptr(self.params), _ptr(self.grads))

    def fwd_bwd(self, frame, embed_index: Sequence[int], color: torch.Tensor, target: torch.Tensor,
                corrected: Optional[torch.Tensor] = None, stream=None):
        """Losses [n_views] and dL/dcolour (same layout as ``color``); gradients of
        the appearance parameters are added to ``self.grads``."""
        nv = frame.frame.n_views
        idx = (ctypes.c_int32 * nv)(*[int(i) for i in embed_index])
        loss = torch.empty(nv, dtype=torch.float32, device=self.device)
        dcol = torch.empty_like(color)
        state = torch.empty(_lib.APPEARANCE_STATE_FLOATS * nv, dtype=torch.float32, device=self.device)
        s = (stream or torch.cuda.current_stream()).cuda_stream
        check(self.lib.gs_appearance_fwd_bwd(ctypes.byref(frame.frame), ctypes.byref(self._c), idx, _ptr(color),
                                             _ptr(target), _ptr(corrected), _ptr(dcol), _ptr(loss), _ptr(state), s),
              "gs_appearance_fwd_bwd")
        self._keep = (state, idx)
        return loss, dcol

    def step(self, lr: float = 1e-2, betas=(0.9, 0.999), eps: float = 1e-8, stream=None):
        self.t += 1
        s = (stream or torch.cuda.current_stream()).cuda_stream
        check(self.lib.gs_adam_step(_ptr(self.params), _ptr(self.grads), _ptr(self.m), _ptr(self.v),
                                    self.params.numel(), lr, betas[0], betas[1], eps, self.t, 1, s),
              "gs_adam_step")


def adam_step(params, grads, m, v, step, lr=1e-2, betas=(0.9, 0.999), eps=1e-8, zero_grads=True, stream=None):
    """Adam on any flat FP32 CUDA tensors (e.g. Gaussian parameters) through gs_adam_step."""
    lib = _lib.load()
    s = (stream or torch.cuda.current_stream()).cuda_stream
    check(lib.gs_adam_step(_ptr(params), _ptr(grads), _ptr(m), _ptr(v), params.numel(), lr, betas[0], betas[1],
                           eps, int(step), int(bool(zero_grads)), s), "gs_adam_step")
