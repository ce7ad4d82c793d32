"""Autotuner of the batched launch (mg_batch_*): chooses, by measurement, the
cluster size (CTAs per team), the target bytes of one FFT tile per problem
size class and the largest Stockham radix per size class, and keeps the
choice in a JSON cache keyed by the batch's shape.

The knobs are the arguments of mg_batch_create.  The search is coordinate
descent from the library's defaults: one knob at a time over its candidate
values, keeping a change only when the measured time per step drops by more
than `min_gain`.  Measuring advances the problems' states, so the tuner saves
every state first and restores it after each trial (mg_set_state with the
saved buffer and centres).

Only argument marshalling and timing happen here; every trial runs the CUDA
batch kernel.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

CLUSTERS = (1, 2, 4, 8)
TILE_TARGETS = (0, 8192, 16384, 32768, 65536)  # 0: the library's default
RADIX_MAX = (0, 2, 4, 8)                         # 0: the library's default
# size classes by points per grid: the knobs are set per class
CLASS_BOUNDS = (8192, 65536)


def size_class(npts):
    for i, b in enumerate(CLASS_BOUNDS):
        if npts <= b:
            return i
    return len(CLASS_BOUNDS)


def signature(shapes, precision, device_name="", extra=""):
    """Cache key of a batch: the multiset of grid shapes, the precision, the
    device and anything else the caller wants to key on."""
    items = sorted(tuple(int(n) for n in s) for s in shapes)
    text = json.dumps({"shapes": items, "precision": int(precision), "device": device_name, "extra": extra})
    return hashlib.sha256(text.encode()).hexdigest()[:32]


def default_settings():
    nc = len(CLASS_BOUNDS) + 1
    return {"cluster": 0, "tile": [0] * nc, "radix": [0] * nc}


def expand(settings, classes):
    """Per-problem tile_bytes and radix_max lists from per-class settings."""
    return ([settings["tile"][c] for c in classes], [settings["radix"][c] for c in classes])


def coordinate_descent(measure, classes_present, min_gain=0.03, clusters=CLUSTERS, tiles=TILE_TARGETS,
                       radices=RADIX_MAX):
    """Search the knobs one at a time.  measure(settings) -> seconds per step
    (float, or None if the setting is rejected).  Returns (best settings,
    best time, list of (settings, time) trials)."""
    trials = []

    def run(s):
        t = measure(s)
        trials.append((json.loads(json.dumps(s)), t))
        return t

    best = default_settings()
    best_t = run(best)
    if best_t is None:
        raise RuntimeError("the default batch settings were rejected")

    def try_values(key, idx, values):
        nonlocal best, best_t
        for v in values:
            cand = json.loads(json.dumps(best))
            if idx is None:
                if cand[key] == v:
                    continue
                cand[key] = v
            else:
                if cand[key][idx] == v:
                    continue
                cand[key][idx] = v
            t = run(cand)
            if t is not None and t < best_t * (1.0 - min_gain):
                best, best_t = cand, t

    try_values("cluster", None, clusters)
    for c in sorted(classes_present):
        try_values("tile", c, tiles)
    for c in sorted(classes_present):
        try_values("radix", c, radices)
    return best, best_t, trials


def load_cache(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def store_cache(path, key, entry):
    d = load_cache(path)
    d[key] = entry
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(d, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def default_cache_path():
    return os.environ.get("MG_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "mgrid", "autotune.json"))


def tune_batch(props, n_steps, dt, scheme, split=0, grid_motion=0, trial_steps=4, cache_path=None,
               retune=False, min_gain=0.03):
    """Settings for a batch of Propagators (same precision and stream), from
    the cache or by measurement.  Returns (settings, per-problem tile_bytes,
    per-problem radix_max, cache entry).  States are left as they were."""
    import numpy as np
    import torch

    from . import capi

    cache_path = cache_path or default_cache_path()
    prec = props[0].precision
    dev = props[0].device
    key = signature([p.N for p in props], prec, torch.cuda.get_device_name(dev), f"{scheme}/{split}/{grid_motion}")
    classes = [size_class(int(np.prod(p.N))) for p in props]
    if not retune:
        entry = load_cache(cache_path).get(key)
        if entry is not None:
            s = entry["settings"]
            tb, rm = expand(s, classes)
            return s, tb, rm, entry

    saved = [(p.psi.clone(),) + tuple(p.get_state(want_psi=False)[1:]) for p in props]
    dts = np.broadcast_to(np.asarray(dt, dtype=np.float64), (len(props),)).copy()

    def restore():
        for p, (u, q, pc, t) in zip(props, saved):
            p.psi.copy_(u)
            p.set_state(None, q, pc, t)

    def measure(s):
        tb, rm = expand(s, classes)
        try:
            b = capi.Batch(props, cluster=s["cluster"], tile_bytes=tb, radix_max=rm)
        except capi.MgError:
            return None
        try:
            b.propagate(1, dts, scheme, split, grid_motion)  # warm-up (graph upload, caches)
            b.sync()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ev[0].record(props[0].stream)
            b.propagate(trial_steps, dts, scheme, split, grid_motion)
            ev[1].record(props[0].stream)
            b.sync()
            return ev[0].elapsed_time(ev[1]) / 1e3 / trial_steps
        except capi.MgError:
            return None
        finally:
            b.close()
            restore()

    t0 = time.time()
    best, best_t, trials = coordinate_descent(measure, set(classes), min_gain=min_gain)
    entry = {"settings": best, "seconds_per_step": best_t, "default_seconds_per_step": trials[0][1],
             "trials": len(trials), "tuning_seconds": time.time() - t0, "n_problems": len(props),
             "trial_steps": trial_steps}
    store_cache(cache_path, key, entry)
    tb, rm = expand(best, classes)
    return best, tb, rm, entry
