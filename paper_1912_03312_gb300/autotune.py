"""Autotuner for the engine's work decomposition.

For one plan it times ``rexi_step`` under candidate settings of
``rexi_plan_set_tiles`` -- points per task for pole items and for shared-cycle
group items, and resident CTAs per SM -- and keeps the fastest.  Results are
cached in a JSON file keyed by device, grid, K, precision, restart length and
orthogonalisation
(``$REXI_AUTOTUNE_CACHE``, default ``~/.cache/rexi_autotune.json``), so a
problem shape is tuned once per machine.  Timing uses CUDA events on the
launch stream; the state is not advanced (the same input is stepped).
"""

from __future__ import annotations

import itertools
import json
import os

import torch

from . import _native as N

DEFAULT_CANDIDATES = {
    "pole_tile": (2048, 1024),
    "group_tile": (512, 1024, 1536, 1792, 2048),
    "ctas_per_sm": (0, 1, 2),
}


# Lanczos plans: group_tile bounds the points of a tile box, ctas_per_sm sets
# the resident CTAs per SM; pole_tile is not used.
LANCZOS_CANDIDATES = {
    "pole_tile": (1024,),
    "group_tile": (512, 768, 1024, 1280, 1536, 1792, 2048),
    "ctas_per_sm": (1, 2),
}


def cache_path():
    return os.environ.get("REXI_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "rexi_autotune.json"))


def _key(plan):
    info = plan.info()
    dev = torch.cuda.get_device_name()
    return "%s|grid=%s|K=%d|prec=%d|m=%d|shared=%d|ortho=%d|window=%d" % (
        dev, "x".join(str(v) for v in reversed(plan.shape)), plan.K, info["precision"], info["restart_m"],
        plan.opts.shared_first_cycle, plan.opts.ortho, plan.opts.window)


def _load():
    try:
        with open(cache_path()) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(d):
    p = cache_path()
    try:
        os.makedirs(os.path.dirname(p), exist_ok=True)
        tmp = p + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, p)
    except OSError:
        pass


def apply(plan, cfg):
    N.check(N.load().rexi_plan_set_tiles(plan.handle, int(cfg["pole_tile"]), int(cfg["group_tile"]),
                                         int(cfg["ctas_per_sm"])), "rexi_plan_set_tiles")


def autotune(plan, psi, candidates=None, steps=3, use_cache=True):
    """Pick and apply the fastest setting for `plan` stepping `psi`; returns
    {"pole_tile", "group_tile", "ctas_per_sm", "ms", "cached"}."""
    key = _key(plan)
    cache = _load() if use_cache else {}
    if key in cache:
        cfg = dict(cache[key])
        apply(plan, cfg)
        cfg["cached"] = True
        return cfg
    cand = candidates or (LANCZOS_CANDIDATES if plan.opts.ortho == 2 else DEFAULT_CANDIDATES)
    stream = torch.cuda.current_stream()
    out = torch.empty_like(psi)
    best = None
    for pt, gt, cps in itertools.product(cand["pole_tile"], cand["group_tile"], cand["ctas_per_sm"]):
        cfg = {"pole_tile": pt, "group_tile": gt, "ctas_per_sm": cps}
        apply(plan, cfg)
        plan.step(psi, out=out)                        # warm-up under this setting
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(steps):
            plan.step(psi, out=out)
        b.record(stream)
        torch.cuda.synchronize()
        ms = a.elapsed_time(b) / steps
        if best is None or ms < best[1]:
            best = (cfg, ms)
    cfg = dict(best[0], ms=best[1])
    apply(plan, cfg)
    if use_cache:
        cache[key] = cfg
        _store(cache)
    cfg["cached"] = False
    return cfg
