"""Autotuner for the force step.

Knobs: the group size n_crit (it changes the host walk, so every candidate
re-walks the tree), packed two-wide FP32 arithmetic or not (packed), target
particles per lane (iblock), list entries per staged tile (tile),
list-split threshold (split) and threads per CTA (block).  Objective: device time of one FP32 force step at fixed theta, the
minimum over repeated CUDA-event timings.  The search is coordinate descent
per n_crit (packed, then iblock, tile, split, block) over the compiled
kernel variants; the winner over all n_crit is cached per GPU name and
workload in tune_cache.json next to this file.

Command line (writes the cache; --out also writes a copy elsewhere):
    python -m paper_1206_1199_gb300.autotune --workload hernquist8m [--out path]
"""
from __future__ import annotations

import argparse
import json
import os

from . import _lib as L

CACHE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tune_cache.json")

# compiled FP32 kernel variants: (block, iblock, tile, packed)
VARIANTS = {(128, 1, 128, 0), (128, 2, 64, 0), (128, 2, 128, 0), (128, 2, 256, 0), (128, 4, 128, 0),
            (128, 4, 256, 0), (64, 2, 128, 0), (64, 4, 128, 0), (256, 2, 128, 0), (256, 1, 128, 0),
            (128, 1, 128, 1), (128, 2, 128, 1), (128, 2, 256, 1), (64, 2, 128, 1), (64, 1, 128, 1),
            (128, 1, 256, 1)}


def workload_key(gpu, w):
    return "%s|%s|n=%d|theta=%g|eps=%g|quad=%d" % (gpu, w.get("model"), int(w.get("n", 0)),
                                                   float(w.get("theta", 0.5)), float(w.get("eps", 0.0)),
                                                   int(bool(w.get("use_quad", True))))


def gpu_name():
    try:
        import torch
        return torch.cuda.get_device_name()
    except Exception:
        return "unknown"


def load_cache(path=CACHE):
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f)
    return {}


def lookup(w, gpu=None):
    """Cached entry {"n_crit", "tune", "ms", ...} for this workload, or None."""
    return load_cache().get(workload_key(gpu or gpu_name(), w))


def cached(w, n_crit_max, gpu=None):
    """Cached Tune for this workload, or None."""
    e = lookup(w, gpu)
    if not e:
        return None
    return L.Tune(**{k: int(v) for k, v in e["tune"].items()})


def _time_step(dev, lists, tune, reps=3, inner=3):
    import torch

    from . import system as S
    n = lists.n_part
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev.bufs["src"].device)
    pot = torch.empty(n, dtype=torch.float64, device=dev.bufs["src"].device)
    S.force(dev, acc, pot, L.OTOO_FP32K, tune)  # also records the graph
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(inner):
            S.force(dev, acc, pot, L.OTOO_FP32K, tune, check=False)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1) / inner)
    return best


def search(pos, mass, w, n_crits=(32, 64, 128, 256), device="cuda", log=print):
    """Coordinate-descent search; returns the best entry and the full table."""
    from . import system as S
    tree = S.Tree(pos, mass, w["leaf_size"])
    table = []
    best = None
    for nc in n_crits:
        lists = tree.lists(w["theta"], nc, w["eps"], w["use_quad"])
        cache = {}

        def run(block, ib, tile, split, packed):
            key = (block, ib, tile, split, packed)
            if key in cache:
                return cache[key]
            if (block, ib, tile, packed) not in VARIANTS:
                cache[key] = float("inf")
                return cache[key]
            tune = L.Tune(block=block, iblock=ib, tile=tile, split=split, ctas_per_sm=0, packed=packed)
            plan = lists.plan(tune)
            dev = S.DeviceSystem.upload(lists, plan, device)
            ms = _time_step(dev, lists, tune)
            del dev
            cache[key] = ms
            row = dict(n_crit=nc, block=block, iblock=ib, tile=tile, split=split, packed=packed, ms=ms,
                       interactions=lists.interactions, groups=lists.n_groups)
            table.append(row)
            log(json.dumps(row))
            return ms

        cur = [128, 2, 128, 4096, 1]
        for pos_k, cands in ((4, (0, 1)), (1, (1, 2, 4)), (2, (64, 128, 256)), (3, (2048, 4096, 8192, 16384)),
                             (0, (64, 128, 256))):
            res = []
            for v in cands:
                c = list(cur)
                c[pos_k] = v
                res.append((run(*c), c))
            cur = min(res)[1]
        ms = run(*cur)
        if best is None or ms < best["ms"]:
            best = dict(n_crit=nc, tune=dict(block=cur[0], iblock=cur[1], tile=cur[2], split=cur[3], ctas_per_sm=0,
                                             packed=cur[4]),
                        ms=ms, interactions=lists.interactions)
    return best, table


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="hernquist8m")
    ap.add_argument("--n-crits", default="32,64,128,256")
    ap.add_argument("--out", default=None)
    args = ap.parse_args()
    from . import ic
    w = dict(ic.WORKLOADS[args.workload])
    pos, mass = ic.make(w["model"], w["n"], w["seed"])
    best, table = search(pos, mass, w, tuple(int(x) for x in args.n_crits.split(",")))
    gpu = gpu_name()
    entry = dict(best, gpu=gpu, workload=args.workload, table=table)
    cache = load_cache()
    cache[workload_key(gpu, w)] = entry
    with open(CACHE, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
    print(json.dumps(dict(best=best)))


if __name__ == "__main__":
    main()
