#!/usr/bin/env python
"""Benchmark of the depth/normal Gaussian rasterizer: ms per forward+backward frame.

One step = one pass of the whole hot path over one frame: per-Gaussian
preprocess, binning (depth sort, pair emission, tile sort, ranges), compositing
forward (colour, alpha, median planar depth, normal), compositing backward and
preprocess backward down to the parameter gradients.

Default workload: the unbounded synthetic scene (3M Gaussians, SH degree 3,
1297x840 pinhole view, FP32), seeded; inputs are larger than L2, so no flush
is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank renders its own replica of the frame (the path needs
no exchange between ranks); ``value`` is the max-over-ranks step time.  The
``reference`` arm times the FP64 CPU oracle on a bounded sample of the same
frame and extrapolates to a whole frame.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per fwd+bwd frame (colour+depth+normal) at 3M Gaussians, 1297x840"
PEAKS_FALLBACK = {"hbm_gbs": 6400.0, "sm_max_mhz": 2032.0}
# The method's own operations per blended (pixel, splat) pair (counted in the
# design notes, section 6): forward 22 FP32 operations (offset 2, quadratic
# form 6, alpha and its clamp 2, alpha test 1, transmittance 2, stop test 1,
# weight 1, colour 3, normal 3, median test 1) and one exp; backward 60 FP32
# operations (alpha recomputed 10, transmittance recovered 2, weight 1,
# colour/normal gradients 6, behind sums 12, dL/dalpha 8, dL/dsigma 1, the
# conic/centre/depth sums 5, their reduction over the pixels 15) plus one exp
# and one reciprocal.  An FMA counts once.
OPS_FWD, OPS_BWD = 22, 60
MUFU_FWD, MUFU_BWD = 1, 2

CONFIGS = {
    "unbounded": dict(workload="unbounded scene, 3M Gaussians, SH deg 3, 1297x840, FP32, fwd+bwd",
                      n=3_000_000, seed=2),
    "object": dict(workload="object scene, 200K Gaussians, SH deg 3, 800x600, FP32, fwd+bwd",
                   n=200_000, seed=1),
    "tiny": dict(workload="tiny scene, 2000 Gaussians, SH deg 0, 128x128, FP32, fwd+bwd", n=2000, seed=0),
}


def make_workload(name):
    from paper_2406_01467_b300 import scenes
    c = CONFIGS[name]
    if name == "unbounded":
        return scenes.unbounded_scene(c["n"], c["seed"]), scenes.unbounded_camera()
    if name == "object":
        return scenes.object_scene(c["n"], c["seed"]), scenes.object_camera()
    return scenes.tiny_scene(c["n"], c["seed"]), scenes.tiny_camera()


def load_traffic(config):
    """DRAM bytes per launch measured by ncu for each stage's kernel, or None for
    a stage whose kernel source changed since the capture (or another workload)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "dram_traffic_unbounded_3M_1297x840.json")
    if config != "unbounded" or not os.path.exists(p):
        return {}
    with open(p) as f:
        d = json.load(f)
    csrc = os.path.join(ROOT, "paper_2406_01467_b300", "csrc")

    def digest(name):
        m = hashlib.sha256()
        for fn in (name, "gs_internal.cuh"):
            with open(os.path.join(csrc, fn), "rb") as fh:
                m.update(fh.read())
        return m.hexdigest()[:16]

    out = {}
    for stage, rec in d["bytes_per_launch"].items():
        if digest(rec["source"]) == d["source_sha256_16"].get(rec["source"]):
            out[stage] = int(rec["bytes"])
    return out


def load_counters(config):
    """Per-launch shared-memory wavefronts of the compositing kernels from the
    committed ncu summary, or {} where the kernel changed since the capture."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "composite_counters_unbounded_3M_1297x840.json")
    if config != "unbounded" or not os.path.exists(p):
        return {}
    with open(p) as f:
        d = json.load(f)
    csrc = os.path.join(ROOT, "paper_2406_01467_b300", "csrc")
    m = hashlib.sha256()
    for fn in ("composite.cu", "gs_internal.cuh"):
        with open(os.path.join(csrc, fn), "rb") as fh:
            m.update(fh.read())
    if m.hexdigest()[:16] != d.get("source_sha256_16"):
        return {}
    return d["per_launch"]


def measure_unit_peaks(device, target_ms=15.0):
    """Peak rates of the units the compositing kernels run on, measured now on
    this GPU with gs_peak_probe (CUDA events, best of 3 launches of about
    target_ms each): FP32 FMAs/s (scalar and packed FP32x2), ex2/s and
    shared-memory bytes/s, with the SM clock sampled meanwhile."""
    import ctypes
    import torch
    from paper_2406_01467_b300 import _lib
    lib = _lib.load()
    sink = torch.zeros(1, device=device)
    stream = torch.cuda.current_stream().cuda_stream
    kinds = (("ffma", _lib.GS_PEAK_FFMA), ("ffma2", _lib.GS_PEAK_FFMA2), ("ex2", _lib.GS_PEAK_EX2),
             ("lds128", _lib.GS_PEAK_LDS128))
    out = {}
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device())
    with sampler:
        for name, kind in kinds:
            work = ctypes.c_int64(0)
            iters = 16
            while True:
                a.record()
                _lib.check(lib.gs_peak_probe(kind, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(work),
                                             ctypes.c_void_p(stream)), "gs_peak_probe")
                b.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                if ms >= target_ms / 4 or iters >= (1 << 22):
                    break
                iters *= 4
            iters = int(min(1 << 24, max(1, iters * target_ms / max(ms, 1e-3))))
            best = None
            for _ in range(3):
                a.record()
                lib.gs_peak_probe(kind, iters, ctypes.c_void_p(sink.data_ptr()), ctypes.byref(work),
                                  ctypes.c_void_p(stream))
                b.record()
                torch.cuda.synchronize()
                ms = a.elapsed_time(b)
                best = ms if best is None else min(best, ms)
            out[name] = work.value / (best * 1e-3)
    clk = sampler.summary(None)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    mhz = clk["sm_mhz"]
    per_clk = {k: round(v / (sms * mhz * 1e6), 2) for k, v in out.items()} if mhz else None
    return {"ffma_per_s": out["ffma"], "ffma2_per_s": out["ffma2"], "ex2_per_s": out["ex2"],
            "lds_bytes_per_s": out["lds128"], "sms": sms, "sm_mhz": mhz, "per_sm_per_clock": per_clk,
            "how": "gs_peak_probe: one resident wave of 8-chain loops per unit, CUDA events, best of 3"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(PEAKS_FALLBACK), "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while it runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self, max_mhz_default):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": max_mhz_default, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def max_over_ranks(value, device):
    """The largest value over all ranks (the value itself without a process group)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def launches_per_step(n_tiles, n_dtypes=1):
    """Kernels libgs launches for one preprocess + bin + fwd + bwd (memsets excluded)."""
    bits = max(1, int(np.ceil(np.log2(max(n_tiles, 2)))))
    tile_passes = (bits + 7) // 8
    setup, pre = 1, n_dtypes
    compaction = 1                    # one-pass compaction (look-back)
    depth_sort = 4                    # one-sweep passes (the compaction counts their digits)
    pair_scan = 1 + 1                 # one-pass pair offsets (look-back), emission
    tile_sort = tile_passes           # one-sweep passes (the emission counts their digits)
    binning = compaction + depth_sort + pair_scan + tile_sort + 1 + 1   # ranges, work order
    # render fwd; backward clear of the visible 2D-gradient rows, composite bwd, preprocess bwd
    return setup + pre + binning + 1 + 2 + n_dtypes


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------
def e2e_pipelined(st, cam, params, capacity, host, n_steps, device):
    """ms per step of the end-to-end loop (parameters uploaded from pinned host
    memory, maps and gradients downloaded to pinned host memory, every step) with
    the copies of neighbouring steps overlapping the compute: two slots of device
    parameters, frame and gradients; an upload stream, a compute stream and a
    download stream ordered by events."""
    import torch
    from paper_2406_01467_b300 import Frame, SceneTensors, scenes
    keys = ("means", "scales", "quats", "opacities", "sh")
    up = [torch.from_numpy(u[0]).to(device) for u in scenes.upstream_grads(11, cam.height, cam.width)]
    slots = []
    for _ in range(2):
        sts = SceneTensors(*(getattr(st, k).clone() for k in keys), st.sh_degree)
        fr = Frame([sts], [(cam, 0)], params, pair_capacity=capacity)
        g = fr.alloc_grads()
        outs = {k: torch.empty(getattr(fr, k).shape, dtype=torch.float32).pin_memory()
                for k in ("color", "alpha", "depth", "normal")}
        gouts = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in g[0].items()}
        ev = {n: torch.cuda.Event() for n in ("h2d", "comp", "d2h")}
        slots.append((sts, fr, g, outs, gouts, ev))
    s_up, s_comp, s_down = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()

    def issue(i):
        sts, fr, g, outs, gouts, ev = slots[i % 2]
        with torch.cuda.stream(s_up):      # the slot's previous compute has read its parameters
            s_up.wait_event(ev["comp"])
            for k in keys:
                getattr(sts, k).copy_(host[k], non_blocking=True)
            ev["h2d"].record(s_up)
        with torch.cuda.stream(s_comp):    # ... and its previous results have been downloaded
            s_comp.wait_event(ev["h2d"])
            s_comp.wait_event(ev["d2h"])
            fr.preprocess()
            fr.bin()
            fr.render()
            fr.backward(*up, grads=g, split=True)
            ev["comp"].record(s_comp)
        with torch.cuda.stream(s_down):
            s_down.wait_event(ev["comp"])
            for k, v in outs.items():
                v.copy_(getattr(fr, k), non_blocking=True)
            for k, v in gouts.items():
                v.copy_(g[0][k], non_blocking=True)
            ev["d2h"].record(s_down)

    for i in range(4):
        issue(i)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    cur = torch.cuda.current_stream()
    a.record(cur)
    for s_ in (s_up, s_comp, s_down):
        s_.wait_stream(cur)
    for i in range(n_steps):
        issue(i)
    for s_ in (s_up, s_comp, s_down):
        cur.wait_stream(s_)
    b.record(cur)
    torch.cuda.synchronize()
    for sl in slots:
        if sl[1].stats().status != 0:
            raise RuntimeError("end-to-end frame status %d" % sl[1].last_status)
    return a.elapsed_time(b) / n_steps


def run_ours(args, rank, world, device):
    import torch
    from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, scenes

    torch.cuda.set_device(device)
    scene, cam = make_workload(args.config)
    st = SceneTensors.from_scene(scene, device)
    params = RenderParams()
    frame = Frame([st], [(cam, 0)], params)
    frame.forward(sync_capacity=True)
    s0 = frame.stats()
    # the pair capacity set to the measured need with a 25% margin (the default
    # of 8 pairs per entry is 4.5x this frame's need), then no host
    # synchronisation inside the timed region
    need = int(s0.n_pairs)
    frame._alloc(int(need * 1.25) + 1024)
    up = [torch.from_numpy(u[0]).to(device) for u in scenes.upstream_grads(11, cam.height, cam.width)]
    grads = frame.alloc_grads()

    n_ev = 6
    def step(ev=None):
        if ev is not None:
            ev[0].record()
        frame.preprocess()
        if ev is not None:
            ev[1].record()
        frame.bin()
        if ev is not None:
            ev[2].record()
        frame.render()
        frame.backward(*up, grads=grads, split=True, events=ev[3:6] if ev is not None else None)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    stats = frame.stats()
    if frame.last_status != 0:
        raise RuntimeError(f"device status {frame.last_status} after warm-up")

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    # the headline: the whole step captured once as a CUDA graph and replayed
    # (every kernel of the step runs in every replay; the graph removes host
    # launch work and inter-kernel gaps)
    from paper_2406_01467_b300 import autotune
    graph = autotune.capture(step)
    for _ in range(args.warmup):
        graph.replay()
    if dist:
        tdist.barrier()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler = ClockSampler(torch.cuda.current_device())
    torch.cuda.synchronize()
    with sampler:
        t0.record()
        for k in range(args.steps):
            graph.replay()
        t1.record()
        torch.cuda.synchronize()
    ms_graph_total = t0.elapsed_time(t1)
    if dist:
        tdist.barrier()
    del graph
    frame.stats()
    if frame.last_status != 0:
        raise RuntimeError(f"device status {frame.last_status} after the timed replays")
    # the same steps launched one kernel at a time, with events between the
    # stages (the per-stage times and rooflines below)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(n_ev)] for _ in range(args.steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    e0.record()
    for k in range(args.steps):
        step(evs[k])
    e1.record()
    torch.cuda.synchronize()
    ms_eager_total = e0.elapsed_time(e1)
    if dist:
        tdist.barrier()
    frame.stats()
    if frame.last_status != 0:
        raise RuntimeError(f"device status {frame.last_status} after the timed steps")
    stages = {"preprocess": 0.0, "bin": 0.0, "render_fwd": 0.0, "composite_bwd": 0.0, "preprocess_bwd": 0.0}
    for ev in evs:
        stages["preprocess"] += ev[0].elapsed_time(ev[1])
        stages["bin"] += ev[1].elapsed_time(ev[2])
        stages["render_fwd"] += ev[2].elapsed_time(ev[3])
        stages["composite_bwd"] += ev[3].elapsed_time(ev[4])
        stages["preprocess_bwd"] += ev[4].elapsed_time(ev[5])
    stages = {k: v / args.steps for k, v in stages.items()}
    ms = max_over_ranks(ms_graph_total / args.steps, device)
    ms_eager = max_over_ranks(ms_eager_total / args.steps, device)

    # ---- end to end: host parameters in, host maps and gradients out --------------------
    e2e = None
    if not args.no_e2e:
        host = {k: getattr(st, k).detach().cpu().pin_memory() for k in ("means", "scales", "quats", "opacities", "sh")}
        outs = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in
                (("color", frame.color), ("alpha", frame.alpha), ("depth", frame.depth), ("normal", frame.normal))}
        gouts = {k: torch.empty(v.shape, dtype=torch.float32).pin_memory() for k, v in grads[0].items()}
        h2d = sum(v.numel() * v.element_size() for v in host.values())
        d2h = sum(v.numel() * v.element_size() for v in outs.values()) + \
            sum(v.numel() * v.element_size() for v in gouts.values())

        def e2e_step():
            for k, v in host.items():
                getattr(st, k).copy_(v, non_blocking=True)
            step()
            for k, v in outs.items():
                v.copy_(getattr(frame, k), non_blocking=True)
            for k, v in gouts.items():
                v.copy_(grads[0][k], non_blocking=True)

        for _ in range(2):
            e2e_step()
        torch.cuda.synchronize()
        n_e2e = max(3, min(args.steps, 20))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(n_e2e):
            e2e_step()
        b.record()
        torch.cuda.synchronize()
        e2e_serial = max_over_ranks(a.elapsed_time(b) / n_e2e, device)
        e2e_ms = e2e_pipelined(st, cam, params, frame.pair_capacity, host, n_e2e, device)
        e2e_ms = max_over_ranks(e2e_ms, device)
        e2e = {"value": round(e2e_ms, 4), "unit": "ms", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": n_e2e, "serial_ms": round(e2e_serial, 4),
               "how": "two slots on three streams: step k+1's parameter upload and step k-1's "
                      "map/gradient download overlap step k's compute"}

    # ---- roofline ---------------------------------------------------------------------------
    peaks, src = load_peaks()
    clocks = sampler.summary(peaks.get("sm_max_mhz", 2032.0))
    K = (scene.sh_degree + 1) ** 2
    N = scene.n
    pbytes = 4 * (3 + 3 + 4 + 1 + 3 * K)
    nvis, P = int(stats.n_visible), int(stats.n_pairs)
    ev_f, ev_b = int(stats.n_evals_fwd), int(stats.n_evals_bwd)
    nbl = int(stats.n_blended)   # (pixel, splat) pairs blended: the compositing's algorithmic unit
    hbm = peaks["hbm_gbs"]
    units = measure_unit_peaks(device)
    # an FMA counts as one operation; the kernels use packed FP32x2 operations
    # where they can, so the FP32 roof is the faster of the two measured rates
    alu_peak = max(units["ffma_per_s"], units["ffma2_per_s"]) / 1e12   # T ops/s
    mufu_peak = units["ex2_per_s"] / 1e12
    gbytes = 4 * (3 + 3 + 4 + 1)          # geometry + opacity of one Gaussian
    shbytes = pbytes - gbytes             # its SH coefficients
    algo = {
        # bytes: geometry + opacity of every Gaussian, SH of the visible ones read;
        # record of the visible ones and rect + key + count of all written
        "preprocess": ("hbm", N * gbytes + nvis * shbytes + nvis * 64 + N * 16),
        # bytes: per pair one read and one write per sort pass lower bound (24 B), depth keys
        "bin": ("hbm", P * 24 + nvis * 16 + N * 8),
        # ops: per blended (pixel, splat) pair (Eq. 3 sums over these); the
        # evaluations the kernels spend on splats that end up not blended are overhead
        "render_fwd": ("alu", (nbl * OPS_FWD, nbl * MUFU_FWD)),
        "composite_bwd": ("alu", (nbl * OPS_BWD, nbl * MUFU_BWD)),
        # bytes: key of every entry, parameters + 2D gradients of visible entries read,
        # all parameter gradients written
        "preprocess_bwd": ("hbm", N * 4 + nvis * (pbytes + 64) + N * pbytes),
    }
    roof = {}
    for k, (bound, work) in algo.items():
        t_s = stages[k] * 1e-3
        if bound == "hbm":
            ach = work / t_s / 1e9
            roof[k] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                       "frac": round(ach / hbm, 4), "bytes": int(work), "ms": round(stages[k], 4)}
        else:
            ops, mufu = work
            a_alu, a_mufu = ops / t_s / 1e12, mufu / t_s / 1e12
            f_alu, f_mufu = a_alu / alu_peak, a_mufu / mufu_peak
            if f_alu >= f_mufu:
                roof[k] = {"bound": "alu", "achieved": round(a_alu, 3), "peak": round(alu_peak, 2),
                           "unit": "Tops/s", "frac": round(f_alu, 4)}
            else:
                roof[k] = {"bound": "mufu", "achieved": round(a_mufu, 3), "peak": round(mufu_peak, 3),
                           "unit": "Tops/s", "frac": round(f_mufu, 4)}
            roof[k].update({"ops": int(ops), "mufu_ops": int(mufu), "ms": round(stages[k], 4),
                            "fp32": {"achieved": round(a_alu, 3), "peak": round(alu_peak, 2), "frac": round(f_alu, 4)},
                            "mufu": {"achieved": round(a_mufu, 4), "peak": round(mufu_peak, 3),
                                     "frac": round(f_mufu, 4)}})
    traffic = load_traffic(args.config)
    for k in roof:
        roof[k]["traffic"] = traffic.get(k)
    # the unit the compositing kernels saturate, from the committed ncu counters of
    # the current sources: shared-memory wavefronts (128 B each) per launch / the
    # live launch time, against the measured shared-memory peak
    counters = load_counters(args.config)
    for k, kern in (("render_fwd", "k_render_fwd"), ("composite_bwd", "k_render_bwd")):
        c = counters.get(kern)
        if c:
            t_s = stages[k] * 1e-3
            sm_bps = c["smem_wavefronts"] * 128 / t_s
            roof[k]["binding"] = {
                "unit": "shared-memory wavefronts (L1 data pipe)",
                "achieved_gbs": round(sm_bps / 1e9, 1), "peak_gbs": round(units["lds_bytes_per_s"] / 1e9, 1),
                "frac": round(sm_bps / units["lds_bytes_per_s"], 4),
                "issue_active": c.get("issue_active"), "source": "ncu wavefronts per launch / event time"}
    # the whole frame: every stage at its own peak, against the measured step
    def t_at_peak(bound, work):
        if bound == "hbm":
            return work / (hbm * 1e9)
        return max(work[0] / (alu_peak * 1e12), work[1] / (mufu_peak * 1e12))
    t_roof = sum(t_at_peak(bound, work) * 1e3 for bound, work in algo.values())
    frame_roof = {"ms_at_peaks": round(t_roof, 4), "frac": round(t_roof / ms, 4),
                  "how": "sum over the stages of algorithmic work / that stage's peak, divided by value"}
    dom = max(stages, key=lambda k: stages[k])
    r = dict(roof[dom])
    r["kernel"] = dom
    r["peak_source"] = (f"HBM: {src} ({'MEASURED_PEAKS.json' if src == 'measured' else 'recipe fallback'}); "
                        "FP32, MUFU and shared memory: measured in this run (unit_peaks)")
    out = {
        "metric": METRIC, "value": round(ms, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms, 4), "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": CONFIGS[args.config]["workload"], "gaussians": N,
                   "image": f"{cam.width}x{cam.height}", "tile": f"{params.tile_w}x{params.tile_h}",
                   "gaussians_per_batch": params.batch,
                   "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas x{world}",
                   "execution": "the step as one CUDA graph, replayed"},
        "ms_per_step_eager": round(ms_eager, 4),
        "roofline": r, "stages": roof, "frame_roofline": frame_roof,
        "counts": {"visible": nvis, "pairs": P, "blended": nbl, "evals_fwd": ev_f, "evals_bwd": ev_b},
        "clocks": clocks, "e2e": e2e, "unit_peaks": units,
        "gpu_launches": launches_per_step(frame_tiles(cam, params)) * args.steps,
        # the timed frame's maps, for the CPU-baseline leg's oracle comparison (not printed)
        "_maps": [m.detach().cpu().numpy() for m in frame.view_maps(0)],
    }
    return out


def frame_tiles(cam, p):
    return ((cam.width + p.tile_w - 1) // p.tile_w) * ((cam.height + p.tile_h - 1) // p.tile_h)


# --------------------------------------------------------------------------------------
# extra lines: BF16 storage under a CUDA graph, the regularised step (Eq. 23-24)
# and the batched many-view frame
# --------------------------------------------------------------------------------------
def timed_graph(step, steps, warmup):
    import torch
    from paper_2406_01467_b300 import autotune
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    eager = autotune.time_step(step, max(3, steps // 4))
    g = autotune.capture(step)
    ms = autotune.time_step(g.replay, steps)
    return ms, eager


def run_bf16(args, device):
    """The 3M scene with every parameter stored in BF16 (FP32 compositing), whole
    forward + backward captured in one CUDA graph."""
    import torch
    from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, autotune, scenes
    scene, cam = make_workload("unbounded")
    st = SceneTensors.from_scene(scene, device, torch.bfloat16)
    fr = Frame([st], [(cam, 0)], RenderParams())
    fr.forward()
    need = int(fr.stats().n_pairs)
    fr._alloc(int(need * 1.25) + 1024)
    up = [torch.from_numpy(u[0]).to(device) for u in scenes.upstream_grads(11, cam.height, cam.width)]
    step = autotune.make_step(fr, up, fr.alloc_grads())
    ms, eager = timed_graph(step, args.steps, args.warmup)
    fr.stats()
    if fr.last_status != 0:
        raise RuntimeError(f"bf16 frame status {fr.last_status}")
    return {"workload": "unbounded scene, 3M Gaussians, BF16 storage, FP32 compositing, 1297x840",
            "ms_per_step_graph": round(ms, 4), "ms_per_step_eager": round(eager, 4),
            "param_bytes": int(sum(getattr(st, k).numel() * 2 for k in ("means", "scales", "quats", "opacities", "sh")))}


def run_batched_bf16(args, device, plain_ms, n_views=4):
    """The precision pattern's headline comparison: several 1297x840 views of the
    3M scene rendered and differentiated together (one launch per kernel, one
    CUDA graph, tile autotuned) with every parameter stored in BF16 and FP32
    compositing, against the plain FP32 single-view step; the same batch with
    FP32 storage separates the two effects."""
    import torch
    from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, autotune, scenes
    scene, _ = make_workload("unbounded")
    views = [(c, 0) for c in scenes.fusion_cameras(n_views, seed=7)]
    out = {"workload": f"unbounded scene, 3M Gaussians, {n_views} views 1297x840 in one frame, fwd+bwd, "
                       "one CUDA graph, autotuned tile and batch", "views": n_views,
           "plain_fp32_single_view_ms": round(plain_ms, 4)}
    for name, dt in (("bf16", torch.bfloat16), ("fp32", torch.float32)):
        st = SceneTensors.from_scene(scene, device, dt)
        params, rep = autotune.tune_tile([st], views, RenderParams(), iters=3, cache_path=None,
                                         candidates=((16, 16), (16, 8), (32, 8)))
        fr = Frame([st], views, params)
        fr.forward()
        need = int(fr.stats().n_pairs)
        fr._alloc(int(need * 1.25) + 1024)
        g = torch.Generator(device=device).manual_seed(13)
        up = [torch.randn(k * fr.n_pixels, device=device, generator=g) for k in (3, 1, 1, 3)]
        step = autotune.make_step(fr, up, fr.alloc_grads())
        ms, eager = timed_graph(step, max(10, args.steps // 4), args.warmup)
        fr.stats()
        if fr.last_status != 0:
            raise RuntimeError(f"batched {name} frame status {fr.last_status}")
        out[name] = {"ms_per_batch_graph": round(ms, 4), "ms_per_view": round(ms / n_views, 4),
                     "ms_per_batch_eager": round(eager, 4), "tile": f"{params.tile_w}x{params.tile_h}",
                     "gaussians_per_batch": params.batch, "autotune_ms": rep["all"], "pairs": need,
                     "param_bytes": int(sum(getattr(st, k).numel() * getattr(st, k).element_size()
                                            for k in ("means", "scales", "quats", "opacities", "sh")))}
        del fr, step, st
        torch.cuda.empty_cache()
    out["bf16_ms_per_view_over_fp32_single_view"] = round(out["bf16"]["ms_per_view"] / plain_ms, 4)
    return out


def run_regularized(args, device, plain_ms):
    """The 3M scene with the depth-distortion (Eq. 23) and normal-consistency
    (Eq. 24) maps rendered and differentiated in the same step, one CUDA graph."""
    import torch
    from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, autotune, scenes
    scene, cam = make_workload("unbounded")
    st = SceneTensors.from_scene(scene, device)
    fr = Frame([st], [(cam, 0)], RenderParams(losses=True))
    fr.forward()
    need = int(fr.stats().n_pairs)
    fr._alloc(int(need * 1.25) + 1024)
    up = [torch.from_numpy(u[0]).to(device) for u in scenes.upstream_grads(11, cam.height, cam.width)]
    up += [torch.from_numpy(u[0]).to(device) for u in scenes.loss_upstream(12, cam.height, cam.width)]
    step = autotune.make_step(fr, up, fr.alloc_grads())
    ms, eager = timed_graph(step, args.steps, args.warmup)
    fr.stats()
    if fr.last_status != 0:
        raise RuntimeError(f"regularised frame status {fr.last_status}")
    return {"workload": "unbounded scene, 3M Gaussians, 1297x840, FP32, colour/alpha/depth/normal + "
                        "L_d (Eq. 23) + L_n (Eq. 24) maps and all six upstream gradients",
            "ms_per_step_graph": round(ms, 4), "ms_per_step_eager": round(eager, 4),
            "overhead_vs_plain_ms": round(ms - plain_ms, 4)}   # both as CUDA graphs


def run_geometry(args, device, n_views=48):
    """Forward-only alpha / depth / normal render of the 3M scene from 48 views
    (1297x840, for fusing depth into a volume), one frame, one CUDA graph; the
    same views through the full forward (colour + backward state) for scale."""
    import torch
    from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, autotune, scenes
    scene, _ = make_workload("unbounded")
    st = SceneTensors.from_scene(scene, device)
    views = [(c, 0) for c in scenes.fusion_cameras(n_views)]
    out = {"workload": f"unbounded scene, 3M Gaussians, {n_views} views 1297x840 in one frame, FP32, forward only",
           "views": n_views}
    for name, p in (("geometry_only", RenderParams(geometry_only=True)), ("full_forward", RenderParams())):
        fr = Frame([st], views, p)
        fr.forward()
        need = int(fr.stats().n_pairs)
        fr._alloc(int(need * 1.15) + 1024)

        def step(fr=fr):
            fr.preprocess()
            fr.bin()
            fr.render()
        ms, eager = timed_graph(step, max(5, args.steps // 20), args.warmup)
        fr.stats()
        if fr.last_status != 0:
            raise RuntimeError(f"{name} frame status {fr.last_status}")
        out[name] = {"ms_per_batch_graph": round(ms, 3), "ms_per_view": round(ms / n_views, 4),
                     "workspace_gb": round(fr.frame.workspace_bytes / 1e9, 2), "pairs": need}
        del fr, step
        torch.cuda.empty_cache()
    return out


def run_filtered(args, device):
    """The paper's default configuration adds the Mip-Splatting 3D filter: its
    variances from 48 views (gs_filter3d) and the 3M step rendered with it."""
    import torch
    from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, autotune, scenes
    scene, cam = make_workload("unbounded")
    st = SceneTensors.from_scene(scene, device)
    views = [(c, 0) for c in scenes.fusion_cameras(48)]
    fv_frame = Frame([st], views, RenderParams(geometry_only=True), pair_capacity=1)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fv_frame.filter3d(0, 0.2, attach=False)
    torch.cuda.synchronize()
    a.record()
    for _ in range(10):
        fv = fv_frame.filter3d(0, 0.2, attach=False)
    b.record()
    torch.cuda.synchronize()
    filt_ms = a.elapsed_time(b) / 10
    del fv_frame
    st.filter_var = fv
    fr = Frame([st], [(cam, 0)], RenderParams())
    fr.forward()
    need = int(fr.stats().n_pairs)
    fr._alloc(int(need * 1.25) + 1024)
    up = [torch.from_numpy(u[0]).to(device) for u in scenes.upstream_grads(11, cam.height, cam.width)]
    step = autotune.make_step(fr, up, fr.alloc_grads())
    ms, eager = timed_graph(step, args.steps, args.warmup)
    fr.stats()
    if fr.last_status != 0:
        raise RuntimeError(f"filtered frame status {fr.last_status}")
    return {"workload": "unbounded scene, 3M Gaussians, 1297x840, FP32, Mip-Splatting 3D filter from 48 views",
            "filter3d_ms_48_views": round(filt_ms, 4), "ms_per_step_graph": round(ms, 4),
            "ms_per_step_eager": round(eager, 4), "pairs": need}


def batched_workload():
    """A 1M-Gaussian unbounded scene seen from 16 orbit views of uneven sizes,
    plus four object scenes (50K/200K/800K/2M) with one 800x600 view each."""
    from paper_2406_01467_b300 import scenes
    big = scenes.unbounded_scene(1_000_000, seed=3)
    objs = [scenes.object_scene(n, seed=5 + i) for i, n in enumerate((50_000, 200_000, 800_000, 2_000_000))]
    views = [(c, 0) for c in scenes.orbit_cameras(16, seed=4)]
    views += [(scenes.object_camera(), 1 + i) for i in range(4)]
    return [big] + objs, views


def run_batched(args, device):
    import torch
    from paper_2406_01467_b300 import Frame, RenderParams, SceneTensors, autotune
    sc, views = batched_workload()
    sts = [SceneTensors.from_scene(x, device) for x in sc]
    params, report = autotune.tune_tile(sts, views, RenderParams(), iters=3, cache_path=None)
    fr = Frame(sts, views, params)
    fr.forward()
    need = int(fr.stats().n_pairs)
    fr._alloc(int(need * 1.25) + 1024)
    g = torch.Generator(device=device).manual_seed(12)
    up = [torch.randn(k * fr.n_pixels, device=device, generator=g) for k in (3, 1, 1, 3)]
    step = autotune.make_step(fr, up, fr.alloc_grads())
    ms, eager = timed_graph(step, max(10, args.steps // 4), args.warmup)
    st = fr.stats()
    if fr.last_status != 0:
        raise RuntimeError(f"batched frame status {fr.last_status}")
    return {"workload": "16 views (512..1600 x 384..1200) of a 1M unbounded scene + 4 object scenes "
                        "(50K/200K/800K/2M, 800x600), FP32, one launch per kernel",
            "views": len(views), "scenes": len(sts), "entries": int(st.n_entries), "pixels": int(fr.n_pixels),
            "pairs": int(st.n_pairs), "tile": f"{params.tile_w}x{params.tile_h}",
            "gaussians_per_batch": params.batch, "autotune_ms": report["all"],
            "ms_per_batch_graph": round(ms, 4), "ms_per_batch_eager": round(eager, 4),
            "ms_per_view_graph": round(ms / len(views), 4)}


# --------------------------------------------------------------------------------------
# CPU oracle (baseline arm and cpu_baseline field)
# --------------------------------------------------------------------------------------
def oracle_step(scene, cam, seed, crop=32, grid=4, collect=None):
    """One step of the CPU oracle on a bounded sample of the frame: its FP32
    binning decisions over all Gaussians, then forward + gradients for grid x
    grid crops of crop x crop pixels, one at a seeded position in each cell of
    a grid x grid partition of the image (stratified, so every step samples
    the whole frame), each restricted to the Gaussians whose rectangles reach
    it.  Returns (estimated ms for the whole frame, seconds spent, sampled
    pixels): binning time + crop time scaled by pixels.  ``collect`` (a list)
    receives (pixels, oracle maps) of every crop."""
    import oracle
    from oracle import binning
    from paper_2406_01467_b300 import scenes

    p = oracle.RenderParams()
    f32 = lambda x: float(np.float32(x))
    p = oracle.RenderParams(lowpass=f32(p.lowpass), alpha_min=f32(p.alpha_min), alpha_max=f32(p.alpha_max),
                            T_min=f32(p.T_min), median_T=f32(p.median_T), clamp_margin=f32(p.clamp_margin))
    t0 = time.perf_counter()
    dec = binning.decide(scene.means, scene.scales, scene.quats, scene.opacities, cam, p)
    t_dec = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    up = [u[0] for u in scenes.upstream_grads(11, cam.height, cam.width)]
    r = dec["rect"]
    t_crop, n_pix = 0.0, 0
    cw, ch = cam.width // grid, cam.height // grid
    for gy in range(grid):
        for gx in range(grid):
            x0 = gx * cw + int(rng.integers(0, max(1, cw - crop)))
            y0 = gy * ch + int(rng.integers(0, max(1, ch - crop)))
            sel = dec["valid"] & (r[:, 1] >= x0) & (r[:, 0] < x0 + crop) & (r[:, 3] >= y0) & (r[:, 2] < y0 + crop)
            sub = scene.subset(np.nonzero(sel)[0])
            ys, xs = np.mgrid[y0:y0 + crop, x0:x0 + crop]
            pix = (ys * cam.width + xs).reshape(-1)
            t1 = time.perf_counter()
            _, _, maps = oracle.render_grads(sub, cam, up, p, pixels=pix)
            t_crop += time.perf_counter() - t1
            if collect is not None:
                collect.append((pix, maps))
            n_pix += len(pix)
    est_ms = (t_dec + t_crop / n_pix * (cam.width * cam.height)) * 1e3
    return est_ms, t_dec + t_crop, n_pix


# The map comparison of the CPU-baseline leg (the parity tests' bar): colour,
# alpha and normal absolute, depth relative; a pixel whose alpha_min / T_min /
# median decisions lie within AMBIG_MARGIN (relative) of their thresholds may
# legitimately go either way in FP32 and is left out.
TOL_ABS, TOL_DEPTH_REL, AMBIG_MARGIN = 1e-4, 1e-4, 2e-4


def oracle_check(collected, gpu_maps):
    """The GPU's maps of the timed frame against the FP64 oracle's on the
    CPU-baseline sample's crops (error maps reduced to their maxima)."""
    c, a, d, n = gpu_maps
    pix = np.concatenate([q for q, _ in collected])
    ref = {k: np.concatenate([m[k] for _, m in collected]) for k in ("color", "alpha", "depth", "normal", "margin")}
    gc, gn = c.reshape(3, -1)[:, pix].T, n.reshape(3, -1)[:, pix].T
    ga, gd = a.reshape(-1)[pix], d.reshape(-1)[pix]
    ok = ref["margin"] >= AMBIG_MARGIN
    ec = np.abs(gc - ref["color"]).max(axis=1)
    ea = np.abs(ga - ref["alpha"])
    en = np.abs(gn - ref["normal"]).max(axis=1)
    ed = np.where(np.abs(ref["depth"]) < 1e-6, np.abs(gd - ref["depth"]),
                  np.abs(gd - ref["depth"]) / np.maximum(np.abs(ref["depth"]), 1e-6))
    bad = ok & ((ec > TOL_ABS) | (ea > TOL_ABS) | (en > TOL_ABS) | (ed > TOL_DEPTH_REL))
    mx = lambda e: float(e[ok].max(initial=0.0))
    return {"pixels": int(len(pix)), "ambiguous_excluded": round(float((~ok).mean()), 5),
            "max_abs_color": mx(ec), "max_abs_alpha": mx(ea), "max_abs_normal": mx(en),
            "max_rel_depth": mx(ed), "outside_tolerance": int(bad.sum()),
            "tolerance": {"abs": TOL_ABS, "depth_rel": TOL_DEPTH_REL, "ambiguity_margin": AMBIG_MARGIN}}


def oracle_baseline(scene, cam, seeds, single_thread=True, gpu_maps=None):
    """The oracle timed on this host over the steps ``seeds`` (oracle_step), and
    once more on one thread.  Both arms of the benchmark use this sample.  With
    ``gpu_maps`` (the timed frame's colour, alpha, depth, normal on the host)
    the first step's oracle maps are also compared with them (oracle_check)."""
    import torch
    cores = torch.get_num_threads()
    collected = [] if gpu_maps is not None else None
    est, secs, pix = zip(*[oracle_step(scene, cam, sd, collect=collected if i == 0 else None)
                           for i, sd in enumerate(seeds)])
    out = {"value": round(float(np.mean(est)), 1), "unit": "ms", "cores": cores, "kind": "oracle",
           "steps": len(seeds), "extrapolated": True, "sampled_pixels_per_step": int(pix[0]),
           "frame_pixels": int(cam.width * cam.height), "seconds": round(float(sum(secs)), 1),
           "sample": f"per step: FP32 binning of all {scene.n} Gaussians + forward and gradients of 16 "
                     f"crops of 32x32 px (one per cell of a 4x4 grid, seeded by the step), the crop time "
                     f"scaled by {cam.width * cam.height}/{pix[0]} pixels",
           "spread_ms": [round(float(min(est)), 1), round(float(max(est)), 1)]}
    if single_thread:
        torch.set_num_threads(1)
        try:
            e1, s1, _ = oracle_step(scene, cam, seeds[0])
        finally:
            torch.set_num_threads(cores)
        out["single_thread_value"] = round(float(e1), 1)
    if collected:
        out["oracle_check"] = oracle_check(collected, gpu_maps)
    return out


def run_reference(args, world):
    scene, cam = make_workload(args.config)
    for k in range(args.warmup):
        oracle_step(scene, cam, 1000 + k)
    base = oracle_baseline(scene, cam, list(range(args.steps)), single_thread=False)
    v = base["value"]
    out = {
        "metric": METRIC, "value": v, "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": v, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "extrapolated": True,
        "sample_seconds_per_step": round(base["seconds"] / args.steps, 2),
        "config": {"workload": CONFIGS[args.config]["workload"], "gaussians": scene.n,
                   "image": f"{cam.width}x{cam.height}", "parallelism": "cpu"},
        "cpu_baseline": base,
        "e2e": {"value": v, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--config", choices=list(CONFIGS), default="unbounded")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the BF16, regularised and batched lines")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, world)), flush=True)
        return 0

    import torch
    if world > 1:
        import torch.distributed as tdist
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    out = run_ours(args, rank, world, f"cuda:{local}")
    gpu_maps = out.pop("_maps", None)
    if not args.no_extras and args.config == "unbounded":
        out["bf16_graph"] = run_bf16(args, f"cuda:{local}")
        out["batched_bf16"] = run_batched_bf16(args, f"cuda:{local}", out["ms_per_step"])
        out["regularized"] = run_regularized(args, f"cuda:{local}", out["ms_per_step"])
        out["filtered"] = run_filtered(args, f"cuda:{local}")
        out["batched"] = run_batched(args, f"cuda:{local}")
        out["geometry_views"] = run_geometry(args, f"cuda:{local}")
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the reference arm's first four steps, plus one on a single thread
        scene, cam = make_workload(args.config)
        out["cpu_baseline"] = oracle_baseline(scene, cam, [0, 1, 2, 3], gpu_maps=gpu_maps)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        tdist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
