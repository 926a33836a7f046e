"""Shared helpers of the parity tests: run the CUDA path and the oracle on the
same seeded inputs and compare."""
from __future__ import annotations

import numpy as np

# Tolerances stated for the FP32 path: colour, alpha and normal absolute, depth relative.
TOL_ABS = 1e-4
TOL_DEPTH_REL = 1e-4
# A pixel whose discrete decisions (alpha >= alpha_min, T' >= T_min, T' <= median_T)
# lie within this relative margin may legitimately go the other way in FP32.
AMBIG_MARGIN = 2e-4


def oracle_params(p):
    """The oracle's RenderParams with the values the library sees (float32)."""
    from oracle import RenderParams as OP
    f = lambda x: float(np.float32(x))
    return OP(lowpass=f(p.lowpass), alpha_min=f(p.alpha_min), alpha_max=f(p.alpha_max),
              T_min=f(p.T_min), median_T=f(p.median_T), clamp_margin=f(p.clamp_margin),
              tile_w=p.tile_w, tile_h=p.tile_h)


def gpu_maps_at(frame, pixels, view=0):
    c, a, d, n = [t.detach().cpu().numpy() for t in frame.view_maps(view)]
    H, W = a.shape
    c = c.reshape(3, -1)[:, pixels].T
    n = n.reshape(3, -1)[:, pixels].T
    return c, a.reshape(-1)[pixels], d.reshape(-1)[pixels], n


def compare_maps(gpu, ref, margin, tol_abs=TOL_ABS, tol_rel=TOL_DEPTH_REL):
    """Returns (ok_mask, report).  Pixels with margin < AMBIG_MARGIN are excluded."""
    gc, ga, gd, gn = gpu
    ok = margin >= AMBIG_MARGIN
    rep = {"ambiguous": float((~ok).mean())}
    ec = np.abs(gc - ref["color"]).max(axis=1)
    ea = np.abs(ga - ref["alpha"])
    en = np.abs(gn - ref["normal"]).max(axis=1)
    ed = np.abs(gd - ref["depth"]) / np.maximum(np.abs(ref["depth"]), 1e-6)
    ed = np.where(np.abs(ref["depth"]) < 1e-6, np.abs(gd - ref["depth"]), ed)
    rep.update(color=float(ec[ok].max(initial=0)), alpha=float(ea[ok].max(initial=0)),
               normal=float(en[ok].max(initial=0)), depth=float(ed[ok].max(initial=0)))
    bad = ok & ((ec > tol_abs) | (ea > tol_abs) | (en > tol_abs) | (ed > tol_rel))
    rep["n_bad"] = int(bad.sum())
    return bad, rep


def _same_ranges(got, ref):
    """Tile ranges agree: identical for non-empty tiles, empty where the oracle's are."""
    got = np.asarray(got, np.int64)
    ref = np.asarray(ref, np.int64)
    full = ref[:, 1] > ref[:, 0]
    np.testing.assert_array_equal(got[full], ref[full])
    assert (got[~full, 1] <= got[~full, 0]).all()


def grad2d_to_record(g2d, pre):
    """dL/d(record field) per entry from the GPU's per-entry 2D sums (the
    `grad2d` debug buffer) and the entries' conic, p and opacity.  The
    compositing backward accumulates sums that are linear in those constants:
    columns (S gs dx, S gs dy, S gs dx^2, S gs dx dy, S gs dy^2, S gs, 0, S sd,
    S sd dx, S sd dy, n1, n2, r, g, b, n0) with gs = dL/dsigma, sd = dL/dd."""
    M = np.asarray(g2d, np.float64)
    c = np.nan_to_num(np.asarray(pre["conic"], np.float64))
    p = np.nan_to_num(np.asarray(pre["p"], np.float64))
    o = np.asarray(pre["opacity"], np.float64)
    safe_o = np.where(o > 0, o, 1.0)
    return {
        "u": c[:, 0] * M[:, 0] + c[:, 1] * M[:, 1] + p[:, 0] * M[:, 7],
        "v": c[:, 1] * M[:, 0] + c[:, 2] * M[:, 1] + p[:, 1] * M[:, 7],
        "conic": np.stack([0.5 * M[:, 2], M[:, 3], 0.5 * M[:, 4]], 1),
        "opacity": np.where(o > 0, -M[:, 5] / safe_o, 0.0),
        "z": M[:, 7],
        "p": M[:, 8:10],
        "n": M[:, [15, 10, 11]],
        "rgb": M[:, 12:15],
    }
