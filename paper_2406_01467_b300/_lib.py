"""ctypes binding of libgs.so (the C ABI declared in include/gs.h).

Argument marshalling only: every stage of the rasterizer runs in the CUDA
library.  Loading fails loudly when the library has not been built; there is
no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, Structure, c_float, c_int32, c_int64, c_size_t, c_void_p

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgs.so")
DEBUG_LIB_PATH = os.path.join(HERE, "libgs_debug.so")   # -DGS_DEBUG: device bounds checks (tests only)

GS_OK, GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA, GS_ERR_TIMEOUT, GS_ERR_NUMERIC, GS_ERR_BOUNDS = range(7)
GS_F32, GS_BF16 = 0, 1
GS_MAX_VIEWS, GS_MAX_SCENES = 64, 16
STATUS_NAMES = {0: "GS_OK", 1: "GS_ERR_INVALID_ARG", 2: "GS_ERR_CAPACITY", 3: "GS_ERR_CUDA",
                4: "GS_ERR_TIMEOUT", 5: "GS_ERR_NUMERIC", 6: "GS_ERR_BOUNDS"}


class GsScene(Structure):
    _fields_ = [("means", c_void_p), ("scales", c_void_p), ("quats", c_void_p),
                ("opacities", c_void_p), ("sh", c_void_p), ("n", c_int64),
                ("sh_degree", c_int32), ("dtype", c_int32), ("filter_var", c_void_p)]


class GsView(Structure):
    _fields_ = [("viewmat", c_float * 16), ("fx", c_float), ("fy", c_float), ("cx", c_float),
                ("cy", c_float), ("width", c_int32), ("height", c_int32),
                ("near_plane", c_float), ("scene", c_int32)]


class GsParams(Structure):
    _fields_ = [("tile_w", c_int32), ("tile_h", c_int32), ("lowpass", c_float),
                ("alpha_min", c_float), ("alpha_max", c_float), ("T_min", c_float),
                ("median_T", c_float), ("clamp_margin", c_float), ("losses", c_int32),
                ("geometry_only", c_int32), ("batch", c_int32)]


class GsFrame(Structure):
    _fields_ = [("scenes", POINTER(GsScene)), ("n_scenes", c_int32),
                ("views", POINTER(GsView)), ("n_views", c_int32), ("params", GsParams),
                ("pair_capacity", c_int64), ("workspace", c_void_p),
                ("workspace_bytes", c_size_t)]


class GsMaps(Structure):
    _fields_ = [("color", c_void_p), ("alpha", c_void_p), ("depth", c_void_p),
                ("normal", c_void_p), ("dist", c_void_p), ("nloss", c_void_p)]


class GsMapGrads(Structure):
    _fields_ = [("dcolor", c_void_p), ("dalpha", c_void_p), ("ddepth", c_void_p),
                ("dnormal", c_void_p), ("ddist", c_void_p), ("dnloss", c_void_p)]


class GsSceneGrads(Structure):
    _fields_ = [("dmeans", c_void_p), ("dscales", c_void_p), ("dquats", c_void_p),
                ("dopacities", c_void_p), ("dsh", c_void_p)]


class GsAppearance(Structure):
    _fields_ = [("n_embeddings", c_int32), ("embed_dim", c_int32), ("hidden", c_int32), ("pad_", c_int32),
                ("params", c_void_p), ("grads", c_void_p)]


APPEARANCE_STATE_FLOATS = 32


class GsStats(Structure):
    _fields_ = [("n_entries", c_int64), ("n_visible", c_int64), ("n_pairs", c_int64),
                ("n_nonfinite", c_int64), ("n_evals_fwd", c_int64), ("n_evals_bwd", c_int64),
                ("n_blended", c_int64), ("status", c_int32)]


EXPORTS = ("gs_workspace_size", "gs_preprocess", "gs_bin", "gs_render_fwd", "gs_render_bwd",
           "gs_composite_bwd", "gs_preprocess_bwd", "gs_filter3d", "gs_appearance_param_count",
           "gs_appearance_fwd_bwd", "gs_adam_step", "gs_debug_copy", "gs_render_fwd_static",
           "gs_check", "gs_debug_wait_timeout", "gs_peak_probe", "gs_debug_checks", "gs_last_error_string")
GS_PEAK_FFMA, GS_PEAK_FFMA2, GS_PEAK_EX2, GS_PEAK_LDS128 = range(4)
STATIC_SCRATCH_BYTES = 32 << 20

_libs = {}   # path -> loaded library


class GsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load libgs.so (or another build of it, e.g. DEBUG_LIB_PATH) and declare
    its prototypes; raises if it is missing."""
    if path in _libs:
        return _libs[path]
    if not os.path.exists(path):
        raise ImportError(f"{os.path.basename(path)} not found at {path}: build it with "
                          f"`python -m paper_2406_01467_b300.build`"
                          f"{' --debug' if path == DEBUG_LIB_PATH else ''}")
    lib = ctypes.CDLL(path)
    pf = POINTER(GsFrame)
    lib.gs_workspace_size.argtypes = [pf]
    lib.gs_workspace_size.restype = c_size_t
    for name in ("gs_preprocess", "gs_bin"):
        getattr(lib, name).argtypes = [pf, c_void_p]
        getattr(lib, name).restype = c_int32
    lib.gs_render_fwd.argtypes = [pf, POINTER(GsMaps), c_void_p]
    lib.gs_render_fwd.restype = c_int32
    lib.gs_render_bwd.argtypes = [pf, POINTER(GsMapGrads), POINTER(GsSceneGrads), c_void_p]
    lib.gs_render_bwd.restype = c_int32
    lib.gs_composite_bwd.argtypes = [pf, POINTER(GsMapGrads), c_void_p]
    lib.gs_composite_bwd.restype = c_int32
    lib.gs_preprocess_bwd.argtypes = [pf, POINTER(GsSceneGrads), c_void_p]
    lib.gs_preprocess_bwd.restype = c_int32
    lib.gs_filter3d.argtypes = [pf, c_int32, c_float, c_void_p, c_void_p]
    lib.gs_filter3d.restype = c_int32
    lib.gs_appearance_param_count.argtypes = [c_int32, c_int32, c_int32]
    lib.gs_appearance_param_count.restype = c_size_t
    lib.gs_appearance_fwd_bwd.argtypes = [pf, POINTER(GsAppearance), c_void_p, c_void_p, c_void_p, c_void_p,
                                          c_void_p, c_void_p, c_void_p, c_void_p]
    lib.gs_appearance_fwd_bwd.restype = c_int32
    lib.gs_adam_step.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p, c_int64, c_float, c_float, c_float,
                                 c_float, c_int32, c_int32, c_void_p]
    lib.gs_adam_step.restype = c_int32
    lib.gs_debug_copy.argtypes = [pf, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                  c_void_p]
    lib.gs_debug_copy.restype = c_int32
    lib.gs_render_fwd_static.argtypes = [pf, POINTER(GsMaps), POINTER(GsStats), c_void_p]
    lib.gs_render_fwd_static.restype = c_int32
    lib.gs_check.argtypes = [pf, POINTER(GsStats), c_void_p]
    lib.gs_check.restype = c_int32
    lib.gs_debug_wait_timeout.argtypes = [pf, c_int32, c_void_p]
    lib.gs_debug_wait_timeout.restype = c_int32
    lib.gs_peak_probe.argtypes = [c_int32, c_int32, c_void_p, POINTER(c_int64), c_void_p]
    lib.gs_peak_probe.restype = c_int32
    lib.gs_last_error_string.argtypes = []
    lib.gs_last_error_string.restype = ctypes.c_char_p
    lib.gs_debug_checks.argtypes = []
    lib.gs_debug_checks.restype = c_int32
    _libs[path] = lib
    return lib


def check(status: int, what: str = "", lib=None):
    """Raise GsError for a non-OK status, with the message of the library that
    returned it (`lib`, default libgs.so)."""
    if status != GS_OK:
        msg = (lib or load()).gs_last_error_string().decode()
        raise GsError(status, f"{what}: {msg}" if what else msg)
