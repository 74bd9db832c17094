"""Learned per-group opening angle.

The paper controls the force error with the accuracy parameter Delta of the
absolute MAC (Section II-B, Eq. SW_MAC; a fraction of the mean force in
Section III-F).  Here a small perceptron predicts, for each group and a
candidate opening angle, the group's RMS relative force error from
statistics of the group's list (list length, minimum cell distance over
cell size, group size over softening, cell mass fraction, group count); the
largest angle whose prediction meets the target is used for that group.

Pipeline (each step runs in libotoo: host walk in C++, forces, direct sums,
network training and inference in CUDA; this module moves data between
the calls):
  snapshots   leap-frog (kick-drift-kick) of the two-polytrope system with
              the method's own FP32 forces at a fixed angle;
  rows        per snapshot, sampled groups x angle grid: features from a
              base walk at theta0, label = log10 of the group's RMS relative
              force error at that angle against the FP64 direct sum on the
              device (otoo_direct);
  training    Adam on the FP32 master weights with the network's own
              forward/backward kernels (bf16 weights in the forward pass);
  selection   otoo_learned_theta on the device over a finer angle grid
              than the training rows' (SELECT_GRID), then a re-walk with one
              angle per group; calibration scales the targets so that the
              selection reaches the target RMS on training snapshots;
  evaluation  learned angles against a fixed angle bisected to the same
              RMS error, and against theta = 0.5.
"""
from __future__ import annotations

import ctypes
import json
import math
import os
import time

import numpy as np

from . import _lib as L
from . import ic
from . import system as S
from .mlp import ThetaNet

THETA_GRID = tuple(round(0.3 + 0.1 * k, 2) for k in range(14))  # 0.3 .. 1.6: angles of the training rows
# angles the selection chooses from (the network takes the angle as an input,
# so it is evaluated between the training angles too): a finer grid lets each
# group come closer to the angle its error budget allows
SELECT_GRID = tuple(round(0.3 + 0.025 * k, 3) for k in range(53))  # 0.3 .. 1.6
THETA0 = 0.9  # angle of the base walk whose list statistics feed the network


def _torch():
    import torch
    return torch


class Evaluator:
    """One particle system: tree, forces at any angle(s), FP64 direct sums."""

    def __init__(self, pos, mass, eps, n_crit=64, leaf_size=8, use_quad=True, device="cuda", tune=None):
        self.pos = np.ascontiguousarray(pos, np.float64)
        self.mass = np.ascontiguousarray(mass, np.float32)
        self.eps, self.n_crit, self.use_quad, self.device = eps, n_crit, use_quad, device
        self.tree = S.Tree(self.pos, self.mass, leaf_size)
        self.tune = tune
        self._src_dev = None

    def lists(self, theta, theta_per_group=None):
        return self.tree.lists(theta, self.n_crit, self.eps, self.use_quad, theta_per_group)

    def force(self, lists, precision=L.OTOO_FP32K, timed=False, on_device=False):
        """Accelerations and potentials in tree order (and the step's ms);
        device tensors when on_device, else host arrays."""
        torch = _torch()
        tune = self.tune or L.default_tune(self.n_crit)
        plan = lists.plan(tune)
        dev = S.DeviceSystem.upload(lists, plan, self.device, use_perm=False)
        n = lists.n_part
        acc = torch.zeros((n, 3), dtype=torch.float64, device=self.device)
        pot = torch.zeros(n, dtype=torch.float64, device=self.device)
        S.force(dev, acc, pot, precision, tune)
        ms = None
        if timed:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(3):
                S.force(dev, acc, pot, precision, tune, check=False)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / 3
        if on_device:
            return acc, pot, ms
        return acc.cpu().numpy(), pot.cpu().numpy(), ms

    def direct(self, targets, on_device=False):
        """FP64 direct sum on the device for tree-order targets (device
        tensors when on_device, else host arrays)."""
        torch = _torch()
        if self._src_dev is None:
            e = self.tree.export()
            src = np.zeros(self.tree.n, dtype=np.dtype(L.Src))
            src["x"], src["y"], src["z"] = e["pos"][:, 0], e["pos"][:, 1], e["pos"][:, 2]
            src["m"] = e["mass"]
            self._src_dev = torch.from_numpy(src.view(np.uint8).reshape(-1).copy()).to(self.device)
        t = torch.from_numpy(np.ascontiguousarray(targets, np.int64)).to(self.device)
        nt = t.shape[0]
        n = self.tree.n
        nch = int(L.load().otoo_direct_chunks(n, nt))
        scratch = torch.empty(4 * nch * nt, dtype=torch.float64, device=self.device)
        acc = torch.empty((nt, 3), dtype=torch.float64, device=self.device)
        pot = torch.empty(nt, dtype=torch.float64, device=self.device)
        status = torch.zeros(1, dtype=torch.int32, device=self.device)
        st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        L.call("otoo_direct", self._src_dev.data_ptr(), n, t.data_ptr(), nt, float(self.eps) ** 2, acc.data_ptr(),
               pot.data_ptr(), scratch.data_ptr(), status.data_ptr(), st)
        torch.cuda.synchronize()
        if int(status.item()) != 0:
            raise L.OtooError(L.OTOO_EDEVICE, "otoo_direct: target index out of range")
        if on_device:
            return acc, pot
        return acc.cpu().numpy(), pot.cpu().numpy()


def relerr(a, ref):
    return np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)


# ---------------------------------------------------------------------------
# snapshots

def leapfrog_snapshots(pos, mass, vel, eps, dt, n_snap, every, theta=0.5, n_crit=64, device="cuda", log=None,
                       resume=None, velocities=None):
    """Kick-drift-kick with the method's FP32 forces at a fixed angle; a
    snapshot (positions) every `every` steps, the first one at step 0.
    resume: (positions, velocities, snapshots so far) of an earlier run's
    last snapshot (load_snapshots) to continue from instead of pos/vel.
    velocities: a list that receives the velocity at each snapshot."""
    if resume is not None:
        x0, v0, done = resume
        x = np.array(x0[-1], np.float64)
        v = np.array(v0[-1], np.float64)
        snaps = [np.array(a) for a in x0]
        vels = [np.array(a) for a in v0]
    else:
        x = np.array(pos, np.float64)
        v = np.array(vel, np.float64)
        snaps, vels = [x.copy()], [v.copy()]

    def accel(xx):
        ev = Evaluator(xx, mass, eps, n_crit, device=device)
        a, _, _ = ev.force(ev.lists(theta))
        out = np.empty_like(a)
        out[ev.tree.export()["perm"]] = a  # back to caller order
        return out

    a = accel(x)
    step = 0
    while len(snaps) < n_snap:
        t0 = time.perf_counter()
        v += 0.5 * dt * a
        x += dt * v
        a = accel(x)
        v += 0.5 * dt * a
        step += 1
        if step % every == 0:
            snaps.append(x.copy())
            vels.append(v.copy())
        if log:
            log("step %d (%.2f s)" % (step, time.perf_counter() - t0))
    if velocities is not None:
        velocities[:] = vels
    return snaps


def save_snapshots(path, snaps, vels, mass, **meta):
    """Checkpoint of a snapshot run: positions and velocities at every
    snapshot (FP64), masses, and the run's parameters (dt, every, eps, ...)."""
    np.savez(path, pos=np.stack(snaps), vel=np.stack(vels), mass=np.asarray(mass, np.float32),
             meta=np.array(json.dumps(meta, sort_keys=True)))


def load_snapshots(path):
    """(positions list, velocities list, masses, parameters) of a checkpoint."""
    d = np.load(path)
    return list(d["pos"]), list(d["vel"]), d["mass"], json.loads(str(d["meta"]))


# ---------------------------------------------------------------------------
# training rows

def group_labels(ev, lists, tgt_dev, ad_dev, off_dev):
    """log10 of each sampled group's RMS relative acceleration error on
    lists (device: otoo_group_rms_error over the groups' targets)."""
    torch = _torch()
    a, _, _ = ev.force(lists, on_device=True)
    at = a.index_select(0, tgt_dev).contiguous()
    ng = off_dev.shape[0] - 1
    out = torch.empty(ng, dtype=torch.float32, device=ev.device)
    status = torch.zeros(1, dtype=torch.int32, device=ev.device)
    L.call("otoo_group_rms_error", at.data_ptr(), ad_dev.data_ptr(), off_dev.data_ptr(), ng, 1e-9, out.data_ptr(),
           status.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    if int(status.item()) != 0:
        raise L.OtooError(L.OTOO_EDEVICE, "otoo_group_rms_error: empty group")
    return out.cpu().numpy()


def group_rows(ev, n_groups, grid=THETA_GRID, theta0=THETA0, seed=0):
    """Rows (features + angle) and labels log10(group RMS relative error) for
    n_groups groups sampled from the base walk at theta0."""
    torch = _torch()
    base = ev.lists(theta0)
    feats = base.features(ev.tree)
    g = base.groups
    rng = np.random.Generator(np.random.PCG64(seed))
    sel = np.sort(rng.choice(base.n_groups, size=min(n_groups, base.n_groups), replace=False))
    # targets: every particle of the sampled groups (tree order), group by group
    tgt = np.concatenate([np.arange(g["first"][k], g["first"][k] + g["count"][k]) for k in sel])
    off = np.concatenate([[0], np.cumsum(g["count"][sel])]).astype(np.int64)
    tgt_dev = torch.from_numpy(tgt.astype(np.int64)).to(ev.device)
    off_dev = torch.from_numpy(off).to(ev.device)
    ad_dev, _ = ev.direct(tgt, on_device=True)
    rows, labels = [], []
    for th in grid:
        tpg = np.full(base.n_groups, -1.0, np.float32)  # negative: the group is skipped
        tpg[sel] = th
        labels.append(group_labels(ev, ev.lists(th, tpg), tgt_dev, ad_dev, off_dev))
        rows.append(np.concatenate([feats[sel], np.full((len(sel), 1), th, np.float32)], 1))
    return np.concatenate(rows).astype(np.float32), np.concatenate(labels).astype(np.float32)


def training_set(snaps, mass, eps, n_crit=64, groups_per_snap=1024, grid=THETA_GRID, theta0=THETA0, device="cuda",
                 log=None):
    X, y = [], []
    for k, x in enumerate(snaps):
        t0 = time.perf_counter()
        ev = Evaluator(x, mass, eps, n_crit, device=device)
        xr, yr = group_rows(ev, groups_per_snap, grid, theta0, seed=1000 + k)
        X.append(xr)
        y.append(yr)
        if log:
            log("snapshot %d: %d rows (%.1f s)" % (k, len(yr), time.perf_counter() - t0))
    return np.concatenate(X), np.concatenate(y)


def train(X, y, steps=3000, lr=3e-3, batch=8192, seed=0, device="cuda", alpha=1.0 / 3.0, beta=1.0 / 3.0,
          theta0=THETA0, grid=THETA_GRID):
    """A network trained on rows X, labels y; it keeps the training rows'
    statistics (standardisation and range), the budget exponents, the base
    walk's angle and the angle grid."""
    net = ThetaNet(None, device, alpha=alpha, beta=beta, theta0=theta0, grid=grid)
    net.fit_scaler(X)
    hist = net.train(X, y, steps=steps, lr=lr, batch=batch, seed=seed, log_every=max(1, steps // 20))
    return net, hist


# ---------------------------------------------------------------------------
# selection and evaluation

def choose_thetas(ev, net, target_rms, grid=None, theta0=None, fallback=0.5, mode="budget"):
    """One opening angle per group (otoo_learned_theta: range check,
    standardisation, budgeted targets, the choice, all on the device) from
    the statistics of a base walk at theta0 (default: the network's).
    mode "equal": every group aims at target_rms; mode "budget": the
    network's budget and calibration."""
    grid = grid if grid is not None else (net.grid or THETA_GRID)
    theta0 = theta0 if theta0 is not None else net.theta0
    base = ev.lists(theta0)
    f = base.features(ev.tree)
    th, _ = net.learned_theta(f, base.groups["count"], grid, target_rms, theta0, fallback, mode)
    return th, base


def calibrate(net, evs, target_rms, n_sub=2048, seed=11, iters=4, log=None):
    """Sets net.calib so that the selection reaches target_rms on the
    snapshots of evs (training data): the RMS relative acceleration error
    over n_sub random particles of each, against the FP64 direct sum, is
    measured for the current calibration and the calibration is scaled by
    target / achieved, iters times.  Returns the achieved RMS per pass."""
    rng = np.random.Generator(np.random.PCG64(seed))
    refs = []
    for ev in evs:
        sub = np.sort(rng.choice(ev.tree.n, size=min(n_sub, ev.tree.n), replace=False))
        refs.append((sub, ev.direct(sub)[0]))
    hist = []
    for _ in range(iters):
        sq, cnt = 0.0, 0
        for ev, (sub, ad) in zip(evs, refs):
            th, _ = choose_thetas(ev, net, target_rms)
            a, _, _ = ev.force(ev.lists(net.theta0, th))
            d = relerr(a[sub], ad)
            sq += float(np.sum(d * d))
            cnt += len(d)
        ach = math.sqrt(sq / cnt)
        hist.append(ach)
        if log:
            log("calibration %.4f: RMS %.4e" % (net.calib, ach))
        net.calib *= target_rms / ach
    return hist


def rms_error(ev, lists, sub, ad, precision=L.OTOO_FP32K, stats=None):
    a, _, ms = ev.force(lists, precision, timed=True)
    d = relerr(a[sub], ad)
    if stats is not None:
        stats.update(p99=float(np.quantile(d, 0.99)), max=float(d.max()))
    return float(np.sqrt(np.mean(d * d))), ms


def compare(ev, net, target_rms=1e-3, n_sub=4096, seed=7, bisect_steps=8, precision_fp64=True, log=None,
            mode="budget"):
    """Learned angles vs fixed angles at equal RMS error (on a subsample)."""
    n = ev.tree.n
    rng = np.random.Generator(np.random.PCG64(seed))
    sub = np.sort(rng.choice(n, size=min(n_sub, n), replace=False))
    ad, _ = ev.direct(sub)
    th, base = choose_thetas(ev, net, target_rms, mode=mode)
    learned = ev.lists(0.5, th)
    st = {}
    e_l, ms_l = rms_error(ev, learned, sub, ad, stats=st)
    res = {"target_rms": target_rms, "mode": mode,
           "learned": dict(st, rms=e_l, ms=ms_l, interactions=learned.interactions, theta_mean=float(th.mean()),
                           theta_min=float(th.min()), theta_max=float(th.max()))}
    l5 = ev.lists(0.5)
    e5, ms5 = rms_error(ev, l5, sub, ad)
    res["fixed_0.5"] = {"rms": e5, "ms": ms5, "interactions": l5.interactions}
    # fixed angle with the learned RMS: bisection on theta, then the
    # interactions and time of the fixed angle interpolated (log-log in the
    # RMS) between the two bisection points that bracket the learned RMS
    lo, hi = 0.05, max(THETA_GRID)
    best = above = None
    for _ in range(bisect_steps):
        mid = 0.5 * (lo + hi)
        lm = ev.lists(mid)
        sm = {}
        em, msm = rms_error(ev, lm, sub, ad, stats=sm)
        if log:
            log("bisect theta %.4f rms %.3e" % (mid, em))
        point = (mid, em, msm, lm.interactions, sm)
        if em > e_l:
            hi = mid
            above = point
        else:
            lo = mid
            best = point
    if best is None:
        lm = ev.lists(lo)
        sm = {}
        em, msm = rms_error(ev, lm, sub, ad, stats=sm)
        best = (lo, em, msm, lm.interactions, sm)
    res["fixed_equal_rms"] = dict(best[4], theta=best[0], rms=best[1], ms=best[2], interactions=best[3])
    if precision_fp64:
        lf = ev.lists(best[0])
        e64, ms64 = rms_error(ev, lf, sub, ad, L.OTOO_FP64)
        res["fp64_equal_rms"] = {"theta": best[0], "rms": e64, "ms": ms64, "interactions": lf.interactions}
    inter_eq, ms_eq = float(best[3]), float(best[2])
    if above is not None and above[1] > best[1] > 0:
        f = math.log(e_l / best[1]) / math.log(above[1] / best[1])
        inter_eq = math.exp(math.log(best[3]) + f * math.log(above[3] / best[3]))
        ms_eq = math.exp(math.log(best[2]) + f * math.log(above[2] / best[2]))
        res["fixed_bracket_above"] = dict(above[4], theta=above[0], rms=above[1], ms=above[2], interactions=above[3])
    res["fixed_interpolated"] = {"rms": e_l, "interactions": inter_eq, "ms": ms_eq}
    res["gain_interactions"] = inter_eq / learned.interactions
    res["gain_time"] = ms_eq / ms_l
    res["gain_interactions_bracket"] = best[3] / learned.interactions
    return res


def merger_ic(n, seed=ic.BASE_SEED + 5):
    pos, mass, vel = ic.polytrope_pair(n, seed, velocities=True)
    return pos, mass, vel


def orbital_period(m_total=1.5, sep=0.05):
    return 2 * math.pi * math.sqrt(sep ** 3 / m_total)


def main():
    import argparse
    ap = argparse.ArgumentParser(description="train the opening-angle network on method-generated snapshots")
    ap.add_argument("--n", type=int, default=1 << 22)
    ap.add_argument("--snaps", type=int, default=16)
    ap.add_argument("--every", type=int, default=5)
    ap.add_argument("--dt-frac", type=float, default=1.0 / 200, help="time step as a fraction of the orbital period")
    ap.add_argument("--groups", type=int, default=1024)
    ap.add_argument("--eps", type=float, default=ic.WORKLOADS["merger4m"]["eps"])
    ap.add_argument("--n-crit", type=int, default=64)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--target", type=float, default=1e-3)
    ap.add_argument("--calib-snaps", type=int, default=4, help="training snapshots the calibration runs on")
    ap.add_argument("--weights", default=None, help="write the trained network here (.npz)")
    ap.add_argument("--summary", default=None, help="write the evaluation here (.json)")
    ap.add_argument("--checkpoint", default=None,
                    help="snapshot checkpoint (.npz): continued when it exists and matches the run, written after")
    ap.add_argument("--recalibrate", action="store_true",
                    help="no training: load --weights, set the selection grid, calibrate, evaluate, write both back")
    args = ap.parse_args()
    log = lambda s: print(s, flush=True)  # noqa: E731
    pos, mass, vel = merger_ic(args.n)
    dt = args.dt_frac * orbital_period()
    meta = dict(n=args.n, dt=dt, every=args.every, eps=args.eps, n_crit=args.n_crit, seed=ic.BASE_SEED + 5)
    resume = None
    if args.checkpoint and os.path.exists(args.checkpoint):
        xs, vs, _, m = load_snapshots(args.checkpoint)
        if m == json.loads(json.dumps(meta, sort_keys=True)):
            resume = (xs[:args.snaps + 1], vs[:args.snaps + 1], len(xs))
            log("checkpoint: %d snapshots loaded" % len(resume[0]))
    t0 = time.perf_counter()
    vels = []
    snaps = leapfrog_snapshots(pos, mass, vel, args.eps, dt, args.snaps + 1, args.every, n_crit=args.n_crit, log=None,
                               resume=resume, velocities=vels)
    if args.checkpoint:
        save_snapshots(args.checkpoint, snaps, vels, mass, **meta)
    t1 = time.perf_counter()
    log("snapshots: %d in %.1f s" % (len(snaps), t1 - t0))
    train_snaps, held_out = snaps[:args.snaps], snaps[args.snaps]
    prev = {}
    if args.recalibrate:
        # the trained network as it is; the rows, losses and times of its
        # training come from the earlier summary
        net = ThetaNet.load(args.weights)
        if args.summary and os.path.exists(args.summary):
            with open(args.summary) as f:
                prev = json.load(f)
        n_rows, hist = prev.get("rows", 0), [prev.get("loss_first", float("nan")), prev.get("loss_last", float("nan"))]
        t2 = t3 = time.perf_counter()
    else:
        X, y = training_set(train_snaps, mass, args.eps, args.n_crit, args.groups, log=log)
        n_rows = int(len(y))
        t2 = time.perf_counter()
        log("rows: %d in %.1f s" % (n_rows, t2 - t1))
        net, hist = train(X, y, steps=args.steps)
        t3 = time.perf_counter()
        log("training: loss %.4g -> %.4g in %.1f s" % (hist[0], hist[-1], t3 - t2))
    net.grid = SELECT_GRID
    net.calib = 1.0
    # calibration on training snapshots spread over the run
    pick = np.unique(np.linspace(0, args.snaps - 1, args.calib_snaps).round().astype(int))
    calib_hist = calibrate(net, [Evaluator(train_snaps[k], mass, args.eps, args.n_crit) for k in pick], args.target,
                           log=log)
    t4 = time.perf_counter()
    if args.weights:
        net.save(args.weights)
    ev = Evaluator(held_out, mass, args.eps, args.n_crit)
    res = compare(ev, net, args.target, log=log, mode="budget")
    res["equal_targets"] = compare(ev, net, args.target, mode="equal", precision_fp64=False)
    times = dict(snapshots=t1 - t0, rows=t2 - t1, training=t3 - t2, calibration=t4 - t3)
    if args.recalibrate:
        times.update({k: v for k, v in prev.get("times_s", {}).items() if k in ("rows", "training")})
    res.update(n=args.n, snapshots=args.snaps, every=args.every, dt=dt, rows=n_rows, loss_first=hist[0],
               loss_last=hist[-1], calib=net.calib, calib_rms=calib_hist, theta0=net.theta0, grid=list(net.grid),
               train_grid=list(THETA_GRID), alpha=net.alpha, beta=net.beta, times_s=times)
    print(json.dumps(res))
    if args.summary:
        with open(args.summary, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
