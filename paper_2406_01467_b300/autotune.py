"""Autotuning of the tile size and the Gaussians-per-batch for a frame
workload, and CUDA-graph capture of a step.

The maps do not depend on the tile size (a pixel's splat list and order are
fixed by the pixel rectangles) nor on the batch (how many records a
compositing warp stages in shared memory per round), so both are pure
performance knobs: smaller tiles give shorter lists and more (tile, splat)
pairs to sort, larger tiles the opposite; larger batches halve the walk's
per-round overhead but double the staging buffers.  ``tune_tile`` times a full
forward + backward step for each (tile, batch) candidate on the actual frame
and caches the winner per (GPU, workload shape) in a JSON file.
"""
from __future__ import annotations

import json
import os
from dataclasses import replace
from typing import Callable, Dict, List, Optional, Sequence, Tuple

import torch

from .rasterize import Frame, RenderParams, SceneTensors

CANDIDATES: Tuple[Tuple[int, int], ...] = ((16, 16), (16, 8), (8, 16), (32, 8), (8, 8), (32, 4), (16, 4))
BATCHES: Tuple[int, ...] = (32, 64)
DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gsr_tile_tuning.json")


def workload_key(scenes: Sequence[SceneTensors], views) -> str:
    """Coarse signature: GPU name, powers of two of the entry and pixel counts,
    view count, SH degrees and dtypes."""
    import math
    name = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
    entries = sum(scenes[v[1] if isinstance(v, tuple) else 0].n for v in views)
    pixels = sum(int(v[0].width if isinstance(v, tuple) else v.width) *
                 int(v[0].height if isinstance(v, tuple) else v.height) for v in views)
    degs = sorted({s.sh_degree for s in scenes})
    dts = sorted({str(s.means.dtype) for s in scenes})
    b = lambda x: int(round(math.log2(max(x, 1))))
    return f"{name}|E2^{b(entries)}|P2^{b(pixels)}|V{len(views)}|deg{degs}|{dts}"


def make_step(frame: Frame, upstream: Sequence[torch.Tensor], grads: List[Dict[str, torch.Tensor]]) -> Callable:
    """One forward + backward pass of ``frame`` with fixed upstream gradients and
    gradient buffers, enqueued on the current stream without host syncs."""
    def step():
        frame.preprocess()
        frame.bin()
        frame.render()
        frame.backward(*upstream, grads=grads, split=True)
    return step


def capture(step: Callable, warmup: int = 2) -> torch.cuda.CUDAGraph:
    """Capture ``step`` into a CUDA graph (after ``warmup`` eager runs on a side stream)."""
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(warmup):
            step()
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    return g


def time_step(step: Callable, iters: int = 5) -> float:
    """Mean ms per call of ``step`` measured with CUDA events."""
    step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(iters):
        step()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / iters


def tune_tile(scenes: Sequence[SceneTensors], views, params: Optional[RenderParams] = None,
              candidates: Sequence[Tuple[int, int]] = CANDIDATES, iters: int = 5,
              cache_path: Optional[str] = DEFAULT_CACHE, upstream=None,
              batches: Sequence[int] = BATCHES) -> Tuple[RenderParams, Dict]:
    """Fastest (tile size, Gaussians-per-batch) for the workload (cached).
    Returns (params, report); the report's ``all`` maps "WxH/bN" to ms."""
    params = params or RenderParams()
    key = workload_key(scenes, views)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            with open(cache_path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if key in cache and "batch" in cache[key]:
        tw, th = cache[key]["tile"]
        return replace(params, tile_w=tw, tile_h=th, batch=cache[key]["batch"]), {"cached": True, **cache[key]}
    report = {}
    best = None
    for (tw, th), nb in [(c, b) for c in candidates for b in batches]:
        p = replace(params, tile_w=tw, tile_h=th, batch=nb)
        fr = Frame(scenes, views, p)
        fr.forward()   # sizes the pair buffer
        need = int(fr.stats().n_pairs)
        if fr.pair_capacity < need * 1.1:
            fr._alloc(int(need * 1.25) + 1024)
        if upstream is None:
            up = [torch.randn(3 * fr.n_pixels, device=fr.device), torch.randn(fr.n_pixels, device=fr.device),
                  torch.randn(fr.n_pixels, device=fr.device), torch.randn(3 * fr.n_pixels, device=fr.device)]
        else:
            up = upstream
        step = make_step(fr, up, fr.alloc_grads())
        ms = time_step(step, iters)
        report[f"{tw}x{th}/b{nb}"] = round(ms, 4)
        if best is None or ms < best[0]:
            best = (ms, tw, th, nb)
        del fr
        torch.cuda.empty_cache()
    entry = {"tile": [best[1], best[2]], "batch": best[3], "ms": round(best[0], 4), "all": report}
    if cache_path:
        cache[key] = entry
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            with open(cache_path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return replace(params, tile_w=best[1], tile_h=best[2], batch=best[3]), {"cached": False, **entry}
