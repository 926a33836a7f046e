"""Python front end of libgs: frames, workspaces and the autograd function.

PyTorch only provides device memory and streams here; every stage of the
rasterizer runs in the CUDA library through the C ABI of include/gs.h.
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass, field
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib
from ._lib import (GS_BF16, GS_ERR_CAPACITY, GS_F32, GS_OK, GsFrame, GsMapGrads, GsMaps, GsParams,
                   GsScene, GsSceneGrads, GsStats, GsView, check)


@dataclass
class RenderParams:
    """Render parameters; defaults follow 3D GS, which the paper keeps (Sec. 4.1.1)."""
    tile_w: int = 16
    tile_h: int = 16
    lowpass: float = 0.3
    alpha_min: float = 1.0 / 255
    alpha_max: float = 0.99
    T_min: float = 1e-4
    median_T: float = 0.5
    clamp_margin: float = 0.15
    losses: bool = False      # keep the per-pixel state of Eq. 23-24 (dist / nloss maps)
    geometry_only: bool = False   # forward-only alpha / depth / normal (no colour, no backward)
    batch: int = 32           # Gaussians a compositing warp stages per round (32 or 64; performance only)

    def to_c(self) -> GsParams:
        return GsParams(self.tile_w, self.tile_h, self.lowpass, self.alpha_min, self.alpha_max,
                        self.T_min, self.median_T, self.clamp_margin, int(bool(self.losses)),
                        int(bool(self.geometry_only)), int(self.batch))


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


@dataclass
class SceneTensors:
    """One set of Gaussians on the device (FP32 or BF16, all arrays the same dtype)."""
    means: torch.Tensor      # (N, 3)
    scales: torch.Tensor     # (N, 3)
    quats: torch.Tensor      # (N, 4) (w, x, y, z)
    opacities: torch.Tensor  # (N,)
    sh: torch.Tensor         # (N, (deg+1)^2, 3)
    sh_degree: int
    filter_var: Optional[torch.Tensor] = None   # (N,) FP32 Mip-Splatting 3D filter variances

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def dtype_code(self) -> int:
        return GS_BF16 if self.means.dtype == torch.bfloat16 else GS_F32

    @staticmethod
    def from_scene(scene, device="cuda", dtype=torch.float32) -> "SceneTensors":
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dtype).contiguous()
        fv = getattr(scene, "filter_var", None)
        fv = None if fv is None else torch.as_tensor(np.ascontiguousarray(fv, np.float32)).to(device)
        return SceneTensors(t(scene.means), t(scene.scales), t(scene.quats), t(scene.opacities),
                            t(scene.sh), int(scene.sh_degree), fv)

    def check(self):
        n = self.n
        K = (self.sh_degree + 1) ** 2
        dt = self.means.dtype
        if dt not in (torch.float32, torch.bfloat16):
            raise TypeError("Gaussian parameters must be float32 or bfloat16")
        shapes = {"means": (n, 3), "scales": (n, 3), "quats": (n, 4), "opacities": (n,),
                  "sh": (n, K, 3)}
        for k, shp in shapes.items():
            a = getattr(self, k)
            if tuple(a.shape) != shp:
                raise ValueError(f"{k} has shape {tuple(a.shape)}, expected {shp}")
            if a.dtype != dt or not a.is_contiguous() or not a.is_cuda:
                raise ValueError(f"{k} must be a contiguous CUDA tensor of dtype {dt}")
        fv = self.filter_var
        if fv is not None and (tuple(fv.shape) != (n,) or fv.dtype != torch.float32 or not fv.is_contiguous()
                               or not fv.is_cuda):
            raise ValueError("filter_var must be a contiguous CUDA float32 tensor of shape (N,)")


def view_struct(cam, scene_index: int = 0) -> GsView:
    v = GsView()
    vm = np.asarray(cam.viewmat, np.float64).reshape(-1)
    for i in range(16):
        v.viewmat[i] = float(vm[i])
    v.fx, v.fy, v.cx, v.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    v.width, v.height = int(cam.width), int(cam.height)
    v.near_plane = float(getattr(cam, "near", 0.2))
    v.scene = int(scene_index)
    return v


class Frame:
    """A batch of views of one or more scenes bound to a workspace.

    ``views`` is a list of (camera, scene_index).  Output maps are allocated
    once; ``forward`` and ``backward`` enqueue the library stages on the current
    stream.  With ``sync_capacity`` the pair count is checked after binning
    (one host synchronisation) and the workspace is grown when needed."""

    def __init__(self, scenes: Sequence[SceneTensors], views, params: RenderParams = None,
                 pair_capacity: Optional[int] = None, lib=None):
        # `lib`: another build of the library (e.g. _lib.load(_lib.DEBUG_LIB_PATH))
        self.lib = lib if lib is not None else _lib.load()
        self.scenes = list(scenes)
        self.views = list(views)
        self.params = params or RenderParams()
        for s in self.scenes:
            s.check()
        self.device = self.scenes[0].means.device
        self._c_scenes = (GsScene * len(self.scenes))()
        self._c_views = (GsView * len(self.views))()
        for i, cv in enumerate(self.views):
            cam, si = cv if isinstance(cv, tuple) else (cv, 0)
            self._c_views[i] = view_struct(cam, si)
        self.sizes = [(int(v.height), int(v.width)) for v in self._c_views]
        self.n_pixels = sum(h * w for h, w in self.sizes)
        self.n_entries = sum(self.scenes[v.scene].n for v in self._c_views)
        self.frame = GsFrame()
        self.frame.scenes = self._c_scenes
        self.frame.n_scenes = len(self.scenes)
        self.frame.views = self._c_views
        self.frame.n_views = len(self.views)
        self.frame.params = self.params.to_c()
        self._bind_scenes()
        cap = pair_capacity if pair_capacity is not None else max(1 << 16, 8 * self.n_entries)
        self._alloc(cap)
        f32 = dict(device=self.device, dtype=torch.float32)
        self.color = None if self.params.geometry_only else torch.empty(3 * self.n_pixels, **f32)
        self.alpha = torch.empty(self.n_pixels, **f32)
        self.depth = torch.empty(self.n_pixels, **f32)
        self.normal = torch.empty(3 * self.n_pixels, **f32)
        self.dist = torch.empty(self.n_pixels, **f32) if self.params.losses else None
        self.nloss = torch.empty(self.n_pixels, **f32) if self.params.losses else None
        self._maps = GsMaps(_ptr(self.color), _ptr(self.alpha), _ptr(self.depth), _ptr(self.normal),
                            _ptr(self.dist), _ptr(self.nloss))

    def _check(self, status, what):
        check(status, what, self.lib)

    def _bind_scenes(self):
        for i, s in enumerate(self.scenes):
            self._c_scenes[i] = GsScene(_ptr(s.means), _ptr(s.scales), _ptr(s.quats), _ptr(s.opacities),
                                        _ptr(s.sh), s.n, s.sh_degree, s.dtype_code, _ptr(s.filter_var))

    def rebind(self, scenes: Sequence[SceneTensors]):
        """Point the frame at new parameter tensors of the same shapes."""
        for a, b in zip(self.scenes, scenes):
            if a.n != b.n or a.sh_degree != b.sh_degree:
                raise ValueError("rebind needs scenes of the same sizes")
            b.check()
        self.scenes = list(scenes)
        self._bind_scenes()

    def _alloc(self, cap: int):
        self.frame.pair_capacity = int(cap)
        self.frame.workspace = None
        self.frame.workspace_bytes = 0
        size = self.lib.gs_workspace_size(ctypes.byref(self.frame))
        if size == 0:
            self._check(_lib.GS_ERR_INVALID_ARG, "gs_workspace_size")
        self.ws = torch.empty(size + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        self.frame.workspace = aligned
        self.frame.workspace_bytes = size
        self.pair_capacity = int(cap)

    # ------------------------------------------------------------------
    def preprocess(self, stream=None):
        self._check(self.lib.gs_preprocess(ctypes.byref(self.frame), _stream(stream)), "gs_preprocess")

    def bin(self, stream=None):
        self._check(self.lib.gs_bin(ctypes.byref(self.frame), _stream(stream)), "gs_bin")

    def render(self, stream=None):
        self._check(self.lib.gs_render_fwd(ctypes.byref(self.frame), ctypes.byref(self._maps),
                                     _stream(stream)), "gs_render_fwd")

    def stats(self, stream=None) -> GsStats:
        st = GsStats()
        self.last_status = self.lib.gs_check(ctypes.byref(self.frame), ctypes.byref(st), _stream(stream))
        return st

    def forward(self, stream=None, sync_capacity: bool = True):
        self.preprocess(stream)
        self.bin(stream)
        if sync_capacity:
            st = self.stats(stream)
            if self.last_status == GS_ERR_CAPACITY:
                self._alloc(int(st.n_pairs * 1.25) + 1024)
                self.preprocess(stream)
                self.bin(stream)
                st = self.stats(stream)
            if self.last_status not in (GS_OK, _lib.GS_ERR_NUMERIC):
                self._check(self.last_status, "binning")
        self.render(stream)

    def filter3d(self, scene: int = 0, scale: float = 0.2, attach: bool = True, stream=None):
        """Mip-Splatting 3D filter variances of ``scene`` from this frame's views of it
        (FP32 (N,)); with ``attach`` the scene renders with them from now on."""
        s = self.scenes[scene]
        out = torch.empty(s.n, dtype=torch.float32, device=self.device)
        self._check(self.lib.gs_filter3d(ctypes.byref(self.frame), int(scene), float(scale), _ptr(out),
                                   _stream(stream)), "gs_filter3d")
        if attach:
            s.filter_var = out
            self._bind_scenes()
        return out

    def alloc_grads(self):
        out = []
        for s in self.scenes:
            f32 = dict(device=self.device, dtype=torch.float32)
            out.append(dict(means=torch.empty((s.n, 3), **f32), scales=torch.empty((s.n, 3), **f32),
                            quats=torch.empty((s.n, 4), **f32), opacities=torch.empty((s.n,), **f32),
                            sh=torch.empty(tuple(s.sh.shape), **f32)))
        return out

    def backward(self, dcolor=None, dalpha=None, ddepth=None, dnormal=None, ddist=None, dnloss=None,
                 grads=None, stream=None, split: bool = False, events=None):
        """Enqueue the backward pass; returns per-scene FP32 gradient dicts.

        ``ddist`` / ``dnloss`` weight the Eq. 23 / Eq. 24 maps (``params.losses``).
        ``split`` issues it as gs_composite_bwd + gs_preprocess_bwd; ``events``
        (three CUDA events) are then recorded before, between and after the two."""
        def flat(t, n):
            if t is None:
                return None
            t = t.reshape(-1)
            if t.numel() != n:
                raise ValueError("upstream gradient has the wrong size")
            return t.to(torch.float32).contiguous()
        dc, da, dd, dn = (flat(dcolor, 3 * self.n_pixels), flat(dalpha, self.n_pixels),
                          flat(ddepth, self.n_pixels), flat(dnormal, 3 * self.n_pixels))
        dl, dq = flat(ddist, self.n_pixels), flat(dnloss, self.n_pixels)
        self._up = (dc, da, dd, dn, dl, dq)   # keep alive until the stream has consumed them
        mg = GsMapGrads(_ptr(dc), _ptr(da), _ptr(dd), _ptr(dn), _ptr(dl), _ptr(dq))
        if grads is None:
            grads = self.alloc_grads()
        cg = (GsSceneGrads * len(self.scenes))()
        for i, g in enumerate(grads):
            cg[i] = GsSceneGrads(_ptr(g["means"]), _ptr(g["scales"]), _ptr(g["quats"]),
                                 _ptr(g["opacities"]), _ptr(g["sh"]))
        self._cg, self._mg = cg, mg
        if not split:
            self._check(self.lib.gs_render_bwd(ctypes.byref(self.frame), ctypes.byref(mg), cg, _stream(stream)),
                  "gs_render_bwd")
            return grads
        if events:
            events[0].record()
        self._check(self.lib.gs_composite_bwd(ctypes.byref(self.frame), ctypes.byref(mg), _stream(stream)),
              "gs_composite_bwd")
        if events:
            events[1].record()
        self._check(self.lib.gs_preprocess_bwd(ctypes.byref(self.frame), cg, _stream(stream)),
              "gs_preprocess_bwd")
        if events:
            events[2].record()
        return grads

    # ------------------------------------------------------------------
    def view_maps(self, v: int = 0):
        """(colour [3,H,W], alpha [H,W], depth [H,W], normal [3,H,W]) of view v
        (colour None for a geometry-only frame)."""
        off = sum(h * w for h, w in self.sizes[:v])
        H, W = self.sizes[v]
        n = H * W
        col = None if self.color is None else self.color[3 * off:3 * (off + n)].view(3, H, W)
        return (col, self.alpha[off:off + n].view(H, W),
                self.depth[off:off + n].view(H, W), self.normal[3 * off:3 * (off + n)].view(3, H, W))

    def loss_maps(self, v: int = 0):
        """(depth distortion [H,W] (Eq. 23), normal consistency [H,W] (Eq. 24)) of view v."""
        if not self.params.losses:
            raise ValueError("the frame was made without params.losses")
        off = sum(h * w for h, w in self.sizes[:v])
        H, W = self.sizes[v]
        return self.dist[off:off + H * W].view(H, W), self.nloss[off:off + H * W].view(H, W)

    def debug_wait_timeout(self, spin_limit: int = 1000, stream=None):
        """Runs the device's bounded-wait test hook (a poll that nothing answers);
        the frame's status then reads GS_ERR_TIMEOUT until the next preprocess."""
        self._check(self.lib.gs_debug_wait_timeout(ctypes.byref(self.frame), int(spin_limit), _stream(stream)),
              "gs_debug_wait_timeout")

    def debug(self):
        """Intermediate buffers (records, rects, sorted pairs, ranges, 2D gradients)."""
        E, P = self.n_entries, self.pair_capacity
        T = sum(((w + self.params.tile_w - 1) // self.params.tile_w) *
                ((h + self.params.tile_h - 1) // self.params.tile_h) for h, w in self.sizes)
        dev = self.device
        rec = torch.zeros((E, 16), dtype=torch.float32, device=dev)
        rect = torch.zeros((E, 4), dtype=torch.int32, device=dev)
        pt = torch.zeros(P, dtype=torch.int32, device=dev)
        pe = torch.zeros(P, dtype=torch.int32, device=dev)
        rg = torch.zeros((T, 2), dtype=torch.int32, device=dev)
        g2 = None if self.params.geometry_only else torch.zeros((E, 16), dtype=torch.float32, device=dev)
        self._check(self.lib.gs_debug_copy(ctypes.byref(self.frame), _ptr(rec), _ptr(rect), _ptr(pt), _ptr(pe),
                                     _ptr(rg), _ptr(g2), _stream(None)), "gs_debug_copy")
        st = self.stats()
        n = int(min(st.n_pairs, P))
        return dict(rec=rec, rect=rect, pair_tile=pt[:n], pair_entry=pe[:n], ranges=rg, grad2d=g2,
                    stats=st)


class _Rasterize(torch.autograd.Function):
    """Differentiable single-view render (Eq. 3, Eq. 4 with the plane of Eq. 13-17,
    Eq. 22): forward = gs_preprocess + gs_bin + gs_render_fwd, backward =
    gs_render_bwd, which replays each pixel's compositing instead of storing
    per-(pixel, splat) state."""

    @staticmethod
    def forward(ctx, means, scales, quats, opacities, sh, frame, sync):
        frame.forward(sync_capacity=sync)
        ctx.frame = frame
        ctx.dtype = means.dtype
        ctx.set_materialize_grads(False)   # unused maps reach the library as NULL (zero)
        c, a, d, n = frame.view_maps(0)
        return c.clone(), a.clone(), d.clone(), n.clone()

    @staticmethod
    def backward(ctx, dc, da, dd, dn):
        frame: Frame = ctx.frame
        g = frame.backward(dc, da, dd, dn)[0]
        cast = lambda t: t if t.dtype == ctx.dtype else t.to(ctx.dtype)
        return (cast(g["means"]), cast(g["scales"]), cast(g["quats"]), cast(g["opacities"]),
                cast(g["sh"]), None, None)


def rasterize(means, scales, quats, opacities, sh, camera, sh_degree: int,
              params: RenderParams = None, pair_capacity: Optional[int] = None,
              frame: Optional[Frame] = None, sync: Optional[bool] = None):
    """Render one view; differentiable w.r.t. all five parameter tensors.

    Returns (colour [3,H,W], alpha [H,W], depth [H,W], normal [3,H,W]); their
    gradients flow to means, scales, quats, opacities and sh (FP32 or BF16, all
    the same dtype), including through the planar depth and the normal.

    ``frame`` reuses the workspace of an earlier call (a Frame of one view whose
    scene has the same size; it is pointed at the new tensors), so a training
    loop allocates nothing per step.  A frame serves one pending backward at a
    time: render, backward, then render again.

    ``sync`` (default: True unless ``pair_capacity`` is given) checks the pair
    count on the host after binning and grows the workspace if needed.  With
    False nothing synchronises, so the call can be captured in a CUDA graph; a
    frame whose pairs exceed the capacity then leaves its maps unwritten, gives
    zero gradients and reports GS_ERR_CAPACITY through ``frame.stats()``."""
    st = SceneTensors(means.detach().contiguous(), scales.detach().contiguous(),
                      quats.detach().contiguous(), opacities.detach().contiguous(),
                      sh.detach().contiguous(), sh_degree)
    if frame is None:
        frame = Frame([st], [(camera, 0)], params, pair_capacity)
    else:
        if len(frame.views) != 1 or len(frame.scenes) != 1:
            raise ValueError("rasterize renders one view of one scene")
        frame.rebind([st])
    if sync is None:
        sync = pair_capacity is None
    return _Rasterize.apply(means, scales, quats, opacities, sh, frame, bool(sync))
