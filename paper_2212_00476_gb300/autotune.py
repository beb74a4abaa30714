"""Autotuner for the launch shapes of libzncc (zncc_set_tuning keys).

For one problem shape (W, H, D, window, iterations, storage) it times the fused path with
CUDA events for candidate values of each knob in turn (coordinate descent, a few rounds),
keeps the fastest, and caches the result in a JSON file keyed by the shape, so that later
runs apply it without searching:

    from paper_2212_00476_gb300 import autotune
    best = autotune.tune(ctx, left, right, disp, sigma_s, sigma_r, iters, storage)

Knobs: the cost kernel's two-blocks-per-SM variant and disparity slices per block
(band-tile depth), the lanes per chunk of the horizontal and vertical DT pairs (disparities
per block = 4 x lanes), the adjacent columns per block of the vertical pairs that store the
volume, how the DT pairs stage their next slices (TMA tensor copies in the horizontal
pairs, cp.async only, or TMA in both directions), and (F16) how the line pairs wait for the
A_hat chain (whole chain before the first, or pass by pass).
"""

from __future__ import annotations

import json
import os
import threading

from . import zncc as Z

CANDIDATES = {
    Z.ZNCC_TUNE_ROW_MINB2: [0, 1],
    Z.ZNCC_TUNE_ROW_SPB: [0, 1, 2, 4, 8],
    Z.ZNCC_TUNE_H_TQ: [0, 2, 4, 8],
    Z.ZNCC_TUNE_V_TQ: [0, 2, 4, 8],
    Z.ZNCC_TUNE_V_LPC: [0, 2],
    Z.ZNCC_TUNE_LINE_LOADS: [0, 1, 2],
    Z.ZNCC_TUNE_AHAT_JOIN: [0, 1, 2],
}
NAMES = {Z.ZNCC_TUNE_ROW_MINB2: "row_minb2", Z.ZNCC_TUNE_ROW_SPB: "row_spb",
         Z.ZNCC_TUNE_H_TQ: "h_tq", Z.ZNCC_TUNE_V_TQ: "v_tq", Z.ZNCC_TUNE_AHAT_SMS: "ahat_sms",
         Z.ZNCC_TUNE_PLANE: "plane", Z.ZNCC_TUNE_PLANE_CS: "plane_cs", Z.ZNCC_TUNE_ROW_LOADS: "row_loads",
         Z.ZNCC_TUNE_V_LPC: "v_lpc", Z.ZNCC_TUNE_LINE_LOADS: "line_loads",
         Z.ZNCC_TUNE_AHAT_JOIN: "ahat_join"}
DEFAULT_CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_build", "autotune.json")
_lock = threading.Lock()


def shape_key(ctx, iters, storage):
    return f"{ctx.W}x{ctx.H}_D{ctx.D}_w{ctx.win}_it{iters}_s{storage}"


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _save(path, data):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    tmp = path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(ctx, settings: dict):
    for name, value in settings.items():
        key = next(k for k, n in NAMES.items() if n == name)
        ctx.set_tuning(key, value)


def _time(ctx, run, reps):
    import torch
    try:
        run()                                   # plan + warm
        torch.cuda.synchronize()
    except Z.ZnccError as e:
        if e.status == Z.ZNCC_EUNSUPPORTED:
            return None
        raise
    stream = ctx.stream or torch.cuda.current_stream()
    times = []
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    times.sort()
    return times[len(times) // 2]


def tune(ctx, left, right, disp, sigma_s, sigma_r, iters, storage=Z.ZNCC_F32, reps=15,
         rounds=2, cache=DEFAULT_CACHE, force=False, log=None):
    """Best knob settings for this shape (cached); leaves them applied to ctx."""
    key = shape_key(ctx, iters, storage)
    with _lock:
        known = _load(cache)
    if not force and key in known:
        apply(ctx, known[key]["settings"])
        return known[key]

    def run():
        ctx.zncc_run(left, right, disp, sigma_s, sigma_r, iters, storage)

    settings = {NAMES[k]: 0 for k in CANDIDATES}
    apply(ctx, settings)
    best_ms = _time(ctx, run, reps)
    for _ in range(rounds):
        changed = False
        for k, values in CANDIDATES.items():
            for v in values:
                if v == settings[NAMES[k]]:
                    continue
                trial = dict(settings)
                trial[NAMES[k]] = v
                apply(ctx, trial)
                ms = _time(ctx, run, reps)
                if log:
                    log(f"{NAMES[k]}={v}: {ms}")
                if ms is not None and ms < best_ms * 0.985:
                    best_ms, settings, changed = ms, trial, True
            apply(ctx, settings)
        if not changed:
            break
    apply(ctx, settings)
    result = {"settings": settings, "ms": best_ms}
    with _lock:
        known = _load(cache)
        known[key] = result
        _save(cache, known)
    return result
