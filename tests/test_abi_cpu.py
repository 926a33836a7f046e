"""The C ABI without a GPU: the library loads, exports every symbol declared in
include/gs.h, and validates arguments on the host (no compute calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2406_01467_b300 import _lib, build, scenes
from paper_2406_01467_b300.rasterize import RenderParams, view_struct

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "gs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z_0-9]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert set(names) == set(_lib.EXPORTS), names
    for n in names:
        assert hasattr(lib, n), n


def _frame(n=100, W=64, H=48, params=None, cap=1000, n_views=1, scene_idx=0):
    sc = (_lib.GsScene * 1)()
    sc[0] = _lib.GsScene(1, 1, 1, 1, 1, n, 3, _lib.GS_F32)   # fake non-null pointers
    vs = (_lib.GsView * n_views)()
    cam = scenes.Camera(np.eye(4), 50.0, 50.0, W / 2, H / 2, W, H)
    for i in range(n_views):
        vs[i] = view_struct(cam, scene_idx)
    f = _lib.GsFrame()
    f.scenes, f.n_scenes, f.views, f.n_views = sc, 1, vs, n_views
    f.params = (params or RenderParams()).to_c()
    f.pair_capacity = cap
    f._keep = (sc, vs)
    return f


def test_workspace_size_grows_with_inputs(lib):
    a = lib.gs_workspace_size(ctypes.byref(_frame(100)))
    b = lib.gs_workspace_size(ctypes.byref(_frame(10_000)))
    c = lib.gs_workspace_size(ctypes.byref(_frame(100, cap=1_000_000)))
    assert 0 < a < b and a < c
    # every extra Gaussian costs at least its record, keys, sort buffers and 2D gradient
    assert (b - a) >= (10_000 - 100) * (64 + 8 + 4 * 6 + 64)


@pytest.mark.parametrize("mut, msg", [
    (lambda f: setattr(f.params, "tile_w", 12), "tile"),
    (lambda f: setattr(f.params, "tile_w", 64), "tile"),
    (lambda f: (setattr(f.params, "tile_w", 64), setattr(f.params, "tile_h", 2)), "tile"),
    (lambda f: setattr(f.params, "alpha_min", 0.0), "alpha_min"),
    (lambda f: setattr(f.params, "alpha_max", 1.0), "alpha_max"),
    (lambda f: setattr(f.params, "median_T", 1.0), "median_T"),
    (lambda f: setattr(f.params, "lowpass", -1.0), "lowpass"),
    (lambda f: setattr(f, "pair_capacity", 0), "pair_capacity"),
    (lambda f: setattr(f, "n_views", 0), "n_views"),
    (lambda f: setattr(f, "n_scenes", 17), "n_scenes"),
    (lambda f: setattr(f.views[0], "scene", 3), "scene index"),
    (lambda f: setattr(f.views[0], "width", 0), "image size"),
    (lambda f: setattr(f.views[0], "fx", -1.0), "intrinsics"),
    (lambda f: setattr(f.views[0], "near_plane", 0.0), "near_plane"),
    (lambda f: setattr(f.scenes[0], "sh_degree", 4), "sh_degree"),
    (lambda f: setattr(f.scenes[0], "dtype", 7), "dtype"),
    (lambda f: setattr(f.scenes[0], "means", None), "NULL"),
    (lambda f: setattr(f.params, "batch", 48), "batch"),
    (lambda f: setattr(f.params, "batch", 128), "batch"),
])
def test_invalid_arguments_are_rejected_on_the_host(lib, mut, msg):
    f = _frame()
    mut(f)
    assert lib.gs_workspace_size(ctypes.byref(f)) == 0
    assert msg in lib.gs_last_error_string().decode()


def test_stage_calls_reject_missing_workspace_without_touching_a_gpu(lib):
    f = _frame()
    st = lib.gs_preprocess(ctypes.byref(f), None)
    assert st == _lib.GS_ERR_INVALID_ARG
    assert "workspace" in lib.gs_last_error_string().decode()
    f.workspace = 256
    f.workspace_bytes = 16
    assert lib.gs_bin(ctypes.byref(f), None) == _lib.GS_ERR_INVALID_ARG
    assert "bytes" in lib.gs_last_error_string().decode()
    f.workspace = 100   # misaligned
    f.workspace_bytes = 1 << 40
    assert lib.gs_render_fwd(ctypes.byref(f), None, None) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_preprocess(None, None) == _lib.GS_ERR_INVALID_ARG


def test_empty_scene_is_valid(lib):
    f = _frame(n=0)
    f.scenes[0] = _lib.GsScene(None, None, None, None, None, 0, 0, _lib.GS_F32)
    assert lib.gs_workspace_size(ctypes.byref(f)) > 0


def test_loss_state_costs_ten_floats_per_pixel(lib):
    a = lib.gs_workspace_size(ctypes.byref(_frame(100, W=64, H=48)))
    b = lib.gs_workspace_size(ctypes.byref(_frame(100, W=64, H=48, params=RenderParams(losses=True))))
    assert b - a >= 10 * 4 * 64 * 48 and b - a < 10 * 4 * 64 * 48 + 512


def test_loss_maps_need_the_loss_state(lib):
    f = _frame()
    f.workspace = 256   # fake, aligned; the check comes before any device work
    f.workspace_bytes = 1 << 40
    maps = _lib.GsMaps(None, None, None, None, 256, None)
    assert lib.gs_render_fwd(ctypes.byref(f), ctypes.byref(maps), None) == _lib.GS_ERR_INVALID_ARG
    assert "losses" in lib.gs_last_error_string().decode()
    mg = _lib.GsMapGrads(None, None, None, None, None, 256)
    assert lib.gs_composite_bwd(ctypes.byref(f), ctypes.byref(mg), None) == _lib.GS_ERR_INVALID_ARG
    assert "losses" in lib.gs_last_error_string().decode()
    f.params.losses = 2
    assert lib.gs_workspace_size(ctypes.byref(f)) == 0


def test_geometry_only_drops_the_backward_state(lib):
    a = lib.gs_workspace_size(ctypes.byref(_frame(1000, W=64, H=48)))
    b = lib.gs_workspace_size(ctypes.byref(_frame(1000, W=64, H=48, params=RenderParams(geometry_only=True))))
    assert a - b >= 12 * 64 * 48 + 64 * 1000
    f = _frame(params=RenderParams(geometry_only=True))
    f.workspace = 256
    f.workspace_bytes = 1 << 40
    maps = _lib.GsMaps(256, None, None, None, None, None)
    assert lib.gs_render_fwd(ctypes.byref(f), ctypes.byref(maps), None) == _lib.GS_ERR_INVALID_ARG
    assert "colour" in lib.gs_last_error_string().decode()
    mg = _lib.GsMapGrads(None, None, None, None, None, None)
    assert lib.gs_composite_bwd(ctypes.byref(f), ctypes.byref(mg), None) == _lib.GS_ERR_INVALID_ARG
    sg = (_lib.GsSceneGrads * 1)()
    assert lib.gs_preprocess_bwd(ctypes.byref(f), sg, None) == _lib.GS_ERR_INVALID_ARG
    assert lib.gs_render_bwd(ctypes.byref(f), ctypes.byref(mg), sg, None) == _lib.GS_ERR_INVALID_ARG
    assert "no backward" in lib.gs_last_error_string().decode()
    f.params.losses = 1
    assert lib.gs_workspace_size(ctypes.byref(f)) == 0


def test_appearance_param_count_and_validation(lib):
    assert lib.gs_appearance_param_count(10, 32, 64) == 10 * 32 + 64 * 32 + 64 + 12 * 64 + 12
    assert lib.gs_appearance_param_count(10, 300, 64) == 0
    assert "embed_dim" in lib.gs_last_error_string().decode()
    f = _frame()
    app = _lib.GsAppearance(2, 8, 8, 0, 256, 256)
    idx = (ctypes.c_int32 * 1)(5)   # out of range: refused before any device work
    st = lib.gs_appearance_fwd_bwd(ctypes.byref(f), ctypes.byref(app), idx, 256, 256, None, None, None, 256, None)
    assert st == _lib.GS_ERR_INVALID_ARG and "embedding index" in lib.gs_last_error_string().decode()
    assert lib.gs_adam_step(256, 256, 256, 256, 10, 0.01, 0.9, 0.999, 1e-8, 0, 1, None) == _lib.GS_ERR_INVALID_ARG


def test_debug_build_reports_its_checks_and_exports_the_same_symbols(lib):
    assert lib.gs_debug_checks() == 0
    build.build(debug=True)
    dbg = _lib.load(_lib.DEBUG_LIB_PATH)
    assert dbg is not lib and dbg.gs_debug_checks() == 1
    for n in _declared_functions():
        assert hasattr(dbg, n), n
