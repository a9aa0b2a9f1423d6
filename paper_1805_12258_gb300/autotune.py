"""Autotuner for the staged kernel: tile width, tile order and launch form
(one CTA per tile, k resident CTAs per SM walking tiles, or the pipelined
ring with its staging depth and consumer groups) for a plane shape; for
batches the launch form (one launch over a packed plane, or launches that
carry each beam's descriptors), tile order and resident CTAs per SM.

Each candidate is timed on the GPU with the plan's kernel events (device time
of the kernel launches only); the best choice is cached in a JSON file keyed
by (templates, levels, dtype, bin-count class) so later runs reuse it.
Cache: $HS_TUNE_CACHE, else ~/.cache/paper_1805_12258_gb300/tune.json.
"""
from __future__ import annotations

import itertools
import json
import math
import os
import threading

import numpy as np

from . import hs

_lock = threading.Lock()

# launch forms: one CTA per tile, resident CTAs walking tiles, pipelined ring
LAUNCH_FORMS = ({"grid_per_sm": 0}, {"grid_per_sm": 3}, {"stages": 3, "z_split": 2},
                {"stages": 3, "z_split": 3})
PLANE_SPACE = {"tile_bins": (64, 96, 128), "order": (1, 2, 3, 4), "launch": LAUNCH_FORMS}
BATCH_SPACE = {"form": ("packed", "beams"), "order": (2, 3, 4), "grid_per_sm": (0, 3)}


def cache_path() -> str:
    p = os.environ.get("HS_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1805_12258_gb300", "tune.json")


def _load():
    try:
        with open(cache_path()) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def _store(key, value):
    with _lock:
        d = _load()
        d[key] = value
        path = cache_path()
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(d, fh, indent=1, sort_keys=True)
        os.replace(tmp, path)


def key_of(kind, n_templates, H, dtype, n_bins):
    return f"{kind}:{n_templates}x{H}:{dtype}:2^{int(round(math.log2(max(1, n_bins))))}"


def _time_plan(fop, ta, n_templates, n_bins, H, dtype, reps, **opts):
    cands = hs.CandBuffer(1 << 16)
    with hs.Plan(n_templates, n_bins, H, ta, dtype=dtype, **opts) as plan:
        if plan.kernel != "staged":
            return math.inf, plan
        for _ in range(2):
            plan.run(fop, cands)
        plan.set_timing(True)
        plan.kernel_time()
        for _ in range(reps):
            plan.run(fop, cands)
        ms, n = plan.kernel_time()
    return ms / max(n, 1), None


def tune_plane(n_templates, n_bins, H, thresholds, *, dtype="f32", fop=None, reps=10,
               use_cache=True, space=None):
    """Best plan options for this shape; returns (options dict, table of
    (options, ms per launch))."""
    import torch
    key = key_of("plane", n_templates, H, dtype, n_bins)
    if use_cache and key in _load():
        return _load()[key]["best"], _load()[key]["table"]
    if fop is None:
        g = torch.Generator(device="cuda")
        g.manual_seed(0)
        fop = torch.empty((n_templates, n_bins), device="cuda").exponential_(generator=g)
        if dtype == "bf16":
            fop = fop.to(torch.bfloat16)
        elif dtype == "f16":
            fop = fop.to(torch.float16)
    space = dict(space or PLANE_SPACE)
    if "grid_per_sm" in space:  # older form of the space: resident CTAs only
        space["launch"] = tuple({"grid_per_sm": g} for g in space.pop("grid_per_sm"))
    table = []
    for tb, order, launch in itertools.product(space["tile_bins"], space["order"],
                                               space["launch"]):
        opts = {"tile_bins": tb, "order": order, **launch}
        try:  # combinations without a compiled kernel are skipped
            ms, _ = _time_plan(fop, thresholds, n_templates, n_bins, H, dtype, reps, **opts)
        except hs.HsError:
            ms = math.inf
        table.append((opts, ms))
    best = min(table, key=lambda x: x[1])[0]
    _store(key, {"best": best, "table": table})
    return best, table


def tune_batch(n_templates, H, thresholds, beams, *, dtype="f32", reps=5, use_cache=True,
               space=None, assume_nonneg=False, packed=None):
    """Best launch form, tile order and resident CTAs per SM for a batch of
    beams [(fop, n_bins, CandBuffer), ...].  packed: (plane, offsets) holding
    the same beams side by side in one plane, to time the single-launch
    form too (skipped when None)."""
    import torch
    n_rep = int(np.median([b[1] for b in beams]))
    key = key_of(f"batch{len(beams)}{'+' if assume_nonneg else ''}", n_templates, H, dtype,
                 n_rep)
    if use_cache and key in _load():
        return _load()[key]["best"], _load()[key]["table"]
    space = dict(space or BATCH_SPACE)
    forms = [f for f in space.get("form", ("beams",)) if f == "beams" or packed is not None]
    table = []
    for form, order, gps in itertools.product(forms, space.get("order", (0,)),
                                              space["grid_per_sm"]):
        with hs.Batch(n_templates, H, thresholds, dtype=dtype, grid_per_sm=gps, order=order,
                      max_beams=len(beams), assume_nonneg=assume_nonneg) as b:
            if form == "packed":
                plane, offs = packed
                b.set_packed(plane, [(o, n, cb) for o, (_, n, cb) in zip(offs, beams)])
            else:
                b.set_beams(beams)
            b.graph_run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                b.graph_run()
            e1.record()
            torch.cuda.synchronize()
            table.append(({"form": form, "order": order, "grid_per_sm": gps},
                          e0.elapsed_time(e1) / reps))
    best = min(table, key=lambda x: x[1])[0]
    _store(key, {"best": best, "table": table})
    return best, table
