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


# Gradients, entry by entry: |gpu - ref| <= GRAD_REL |ref| + GRAD_SPREAD spread
# + GRAD_FLOOR max|ref|, where ref is the FP64 oracle and spread the largest
# change of that entry over FP32 evaluations of the oracle (oracle.fp32_spread).
# The relative 1e-3 alone is out of reach of any FP32 evaluation on the entries
# that are sums of cancelling terms or that pass through a nearly singular
# conic: the oracle's own FP32 evaluation misses it on about 1% of them.
GRAD_REL = 1e-3
GRAD_SPREAD = 16.0
GRAD_FLOOR = 1e-9


def grad_report(g_gpu, g_ref, spread=None, rel=GRAD_REL, c_spread=GRAD_SPREAD, floor=GRAD_FLOOR):
    """Per-entry comparison of gradient arrays (dicts of arrays).

    Returns {name: dict(n, bad, worst, worst_index, worst_ref, norm)}: ``bad``
    entries miss the bound above (without ``spread``: |gpu - ref| <= rel |ref|
    on entries above 1e-6 of the largest); ``worst`` is the largest ratio of an
    entry's difference to its bound; ``norm`` = ||gpu - ref|| / ||ref||."""
    out = {}
    for k in g_ref:
        a = np.asarray(g_gpu[k], np.float64).reshape(-1)
        b = np.asarray(g_ref[k], np.float64).reshape(-1)
        assert a.shape == b.shape, (k, a.shape, b.shape)
        scale = np.abs(b).max(initial=0.0)
        err = np.abs(a - b)
        if spread is None:
            sel = np.abs(b) > 1e-6 * scale
            bound = np.where(sel, rel * np.abs(b), np.inf)
        else:
            bound = rel * np.abs(b) + c_spread * np.asarray(spread[k], np.float64).reshape(-1) + floor * scale
        r = err / np.where(bound > 0, bound, 1e-300)
        i = int(np.argmax(r)) if len(r) else 0
        out[k] = dict(n=int(np.isfinite(bound).sum()), bad=int((err > bound).sum()),
                      worst=float(r[i]) if len(r) else 0.0, worst_index=i,
                      worst_ref=float(b[i]) if len(b) else 0.0,
                      norm=float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)))
    return out


def assert_grads_close(g_gpu, g_ref, spread=None, what="", **kw):
    """Fails unless every entry of every array is within its bound (grad_report)
    and each array's relative norm error is within GRAD_REL."""
    rep = grad_report(g_gpu, g_ref, spread, **kw)
    bad = {k: v for k, v in rep.items() if v["bad"] or v["norm"] > kw.get("rel", GRAD_REL)}
    assert not bad, f"{what}: {bad}"
    assert any(v["n"] for v in rep.values()), f"{what}: nothing to compare"
    return rep


def oracle_grads_with_spread(scene, cam, up, op, pixels=None, fn=None):
    """FP64 oracle gradients of the parameters and of the 2D quantities for the
    upstream maps ``up``, and their FP32 spreads (oracle.fp32_spread).
    Returns (param_grads, grads2d, param_spread, grads2d_spread).  ``fn(scene)``
    replaces oracle.render_grads (it must return the same first two items)."""
    import oracle

    def grads(s):
        pg, g2 = (fn(s) if fn else oracle.render_grads(s, cam, up, op, pixels=pixels))[:2]
        return {**pg, **{"2d." + k: v for k, v in g2.items()}}

    ref, spread = oracle.fp32_spread(grads, scene)

    def split(d):
        return ({k: v for k, v in d.items() if not k.startswith("2d.")},
                {k[3:]: v for k, v in d.items() if k.startswith("2d.")})

    (pg, g2), (sp, s2) = split(ref), split(spread)
    return pg, g2, sp, s2
