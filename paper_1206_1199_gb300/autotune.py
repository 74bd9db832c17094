"""Autotuner for the force kernel: block size, target particles per thread,
tile length, list-split threshold, resident CTAs per SM, and (with a re-walk
on the host) the group size n_crit.  Objective: device time of one force
step at fixed theta.  Results are cached per GPU name and workload in
tune_cache.json next to this file."""
from __future__ import annotations

import json
import os

from . import _lib as L

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")


def _key(gpu, w):
    return "%s|%s|n=%d|theta=%g|quad=%d" % (gpu, w.get("model"), int(w.get("n", 0)), float(w.get("theta", 0.5)),
                                            int(bool(w.get("use_quad", True))))


def _gpu_name():
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def load_cache():
    if os.path.exists(CACHE):
        with open(CACHE) as f:
            return json.load(f)
    return {}


def cached(w, n_crit_max, gpu=None):
    """Cached tuning for this workload (None if absent or not valid for
    the largest group)."""
    entry = load_cache().get(_key(gpu or _gpu_name(), w))
    if not entry:
        return None
    t = L.Tune(**{k: int(v) for k, v in entry["tune"].items()})
    if t.block * t.iblock < n_crit_max:
        return None
    return t
