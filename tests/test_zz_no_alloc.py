"""gs_render_fwd_static: the forward render for callers that cannot allocate
device memory (plugins inside an application that owns the allocator,
real-time loops that forbid allocation).  Its workspace is a device array
inside the library; the test checks, through the C ABI, that two calls in a row
give the same maps as the ordinary path with a caller-allocated workspace, and
that a frame too big for the array is refused before any GPU work.

Kept in a file of its own, collected last, so that a run that stops at the
first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, _lib, build, scenes
from paper_2406_01467_b300.rasterize import view_struct


def _c_frame(st: SceneTensors, cam, params: RenderParams, cap: int):
    sc = (_lib.GsScene * 1)()
    sc[0] = _lib.GsScene(st.means.data_ptr(), st.scales.data_ptr(), st.quats.data_ptr(),
                         st.opacities.data_ptr(), st.sh.data_ptr(), st.n, st.sh_degree, st.dtype_code)
    vs = (_lib.GsView * 1)()
    vs[0] = view_struct(cam, 0)
    f = _lib.GsFrame()
    f.scenes, f.n_scenes, f.views, f.n_views = sc, 1, vs, 1
    f.params = params.to_c()
    f.pair_capacity = cap
    f.workspace, f.workspace_bytes = None, 0
    f._keep = (sc, vs)
    return f


def test_oversized_frame_is_refused_with_both_sizes():
    build.build()
    lib = _lib.load()
    f = _c_frame_fake(n=2_000_000, W=1024, H=1024, cap=10_000_000)
    out = _lib.GsMaps(1, 1, 1, 1)
    st = lib.gs_render_fwd_static(ctypes.byref(f), ctypes.byref(out), None, None)
    assert st == _lib.GS_ERR_INVALID_ARG
    msg = lib.gs_last_error_string().decode()
    assert "static scratch holds" in msg and str(_lib.STATIC_SCRATCH_BYTES) in msg


def _c_frame_fake(n, W, H, cap):
    """A frame with placeholder device pointers: only host-side sizing runs."""
    sc = (_lib.GsScene * 1)()
    sc[0] = _lib.GsScene(1, 1, 1, 1, 1, n, 3, _lib.GS_F32)
    vs = (_lib.GsView * 1)()
    vs[0] = view_struct(scenes.Camera(np.eye(4), 500.0, 500.0, W / 2, H / 2, W, H), 0)
    f = _lib.GsFrame()
    f.scenes, f.n_scenes, f.views, f.n_views = sc, 1, vs, 1
    f.params = RenderParams().to_c()
    f.pair_capacity = cap
    f._keep = (sc, vs)
    return f


@pytest.mark.gpu
def test_static_scratch_forward_matches_caller_workspace_twice():
    lib = _lib.load()
    p = RenderParams()
    cases = [(scenes.tiny_scene(2000, seed=0), scenes.tiny_camera()),
             (scenes.object_scene(20_000, seed=4), scenes.object_camera(320, 240, 440.0))]
    for sc, cam in cases:       # two calls in a row, different frames
        st = SceneTensors.from_scene(sc, "cuda")
        ref = Frame([st], [(cam, 0)], p)
        ref.forward()
        cap = int(ref.stats().n_pairs) + 1024
        f = _c_frame(st, cam, p, cap)
        npix = cam.width * cam.height
        outs = [torch.full((k * npix,), -1.0, device="cuda") for k in (3, 1, 1, 3)]
        maps = _lib.GsMaps(*[o.data_ptr() for o in outs])
        stats = _lib.GsStats()
        status = lib.gs_render_fwd_static(ctypes.byref(f), ctypes.byref(maps), ctypes.byref(stats),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert status == _lib.GS_OK, lib.gs_last_error_string().decode()
        assert stats.n_pairs == ref.stats().n_pairs and stats.n_visible == ref.stats().n_visible
        assert stats.n_evals_bwd == 0 and stats.status == _lib.GS_OK   # no backward ran in this call
        for got, want in zip(outs, (ref.color, ref.alpha, ref.depth, ref.normal)):
            # same kernels on the same inputs: within the parity tolerance (in fact equal)
            torch.testing.assert_close(got, want, rtol=0, atol=1e-6)
