"""Force-step benchmark: softened gravity of every group against its shared
interaction list on one GB300 (interactions per second and ms per step).

Default workload: Hernquist halo N = 2^23 (a = 1, truncated at 100 a), eps
5e-4, theta 0.5, quadrupole cells, FP32 centre-relative pairs with Kahan
sums (FP64 form timed beside it).  A step is one otoo_force call (CUDA graph:
ticket reset, persistent force kernel, chunk merge) over device-resident
groups and lists; the host tree and walk are built once before timing.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(the only reference this method has) on a bounded sample of the same
workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FP32_LANES_PER_SM = 128  # FP32 FMA lanes per SM (4 partitions x 32)

# DRAM bytes of one force-kernel launch (dram__bytes_read.sum +
# dram__bytes_write.sum, one ncu capture of k_force_warp2<4,2,8> on the
# Hernquist N = 2^23 workload: 27.42 GB + 0.673 GB, softened quadrupole with
# 80-byte cell records), keyed by the workload, n_crit and tuning it was
# taken on; other configurations report null.
CAPTURED_TRAFFIC = {("hernquist8m", 8388608, 128, (128, 2, 256, 8192, 1)): 27418532096 + 672520192}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="hernquist8m")
    ap.add_argument("--n", type=int, default=0, help="override particle count (testing only)")
    ap.add_argument("--n-crit", type=int, default=0)
    ap.add_argument("--tune", default="", help="block,iblock,tile,split[,packed] (default: autotuner cache)")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--err-targets", type=int, default=512)
    ap.add_argument("--cpu-fraction", type=float, default=1.0 / 16,
                    help="share of the workload's groups in the CPU oracle's seeded sample (both arms)")
    ap.add_argument("--cpu-repeats", type=int, default=3, help="timed repeats of the CPU sample (this arm)")
    ap.add_argument("--skip-extras", action="store_true",
                    help="skip the batched 64-system step and the learned-angle comparison")
    ap.add_argument("--skip-walk", action="store_true", help="skip the device-walk step")
    ap.add_argument("--skip-sw", action="store_true", help="skip the absolute-MAC (delta) sweep")
    ap.add_argument("--skip-step", action="store_true", help="skip the whole step on the device")
    ap.add_argument("--skip-sph", action="store_true", help="skip the SPH density stage")
    ap.add_argument("--fused-only", action="store_true",
                    help="only the walk fused with the force against the split device step, on this workload")
    ap.add_argument("--walk-group-set", type=int, default=0,
                    help="groups one warp walks together in the device walks (1..8; 0: chosen by the library)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cores():
    return len(os.sched_getaffinity(0))


def workload(args, rank=0):
    from paper_1206_1199_gb300 import ic
    w = dict(ic.WORKLOADS[args.workload])
    if args.n:
        w["n"] = args.n
    if args.n_crit:
        w["n_crit"] = args.n_crit
    # independent problems per rank (weak scaling): rank r draws seed + 100 r
    w["seed"] = w["seed"] + 100 * rank
    pos, mass = ic.make(w["model"], w["n"], w["seed"])
    return w, pos, mass


def pick_tune(w, args):
    """The autotuner's cached choice for this GPU and workload (it sets
    n_crit), else the default tuning at the workload's n_crit."""
    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import autotune
    if getattr(args, "tune", None):
        v = [int(x) for x in args.tune.split(",")]
        packed = v[4] if len(v) > 4 else 0
        return L.Tune(block=v[0], iblock=v[1], tile=v[2], split=v[3], ctas_per_sm=0, packed=packed), "given"
    entry = None if args.n_crit else autotune.lookup(w)
    if entry:
        w["n_crit"] = int(entry["n_crit"])
        return L.Tune(**{k: int(v) for k, v in entry["tune"].items()}), "autotuned"
    return L.default_tune(w["n_crit"]), "default"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "otoo_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=clocks.sm,clocks.max.sm,power.draw,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        return {"sm_mhz": float(np.median([r[0] for r in rows])), "sm_max_mhz": rows[0][1], "reasons": reasons,
                "samples": len(rows)}


def max_over_ranks(value, device="cpu"):
    """Largest value over the ranks of the default process group (the value
    itself without one)."""
    import torch
    import torch.distributed as tdist
    if not (tdist.is_available() and tdist.is_initialized()) or tdist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Whole-job throughput of weak scaling: every rank processes its own
    units, the job takes the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def rel_err(a, ref):
    d = np.linalg.norm(a - ref, axis=1) / np.linalg.norm(ref, axis=1)
    return float(np.sqrt(np.mean(d * d))), float(d.max())


def run_ours(args):
    import torch
    import torch.distributed as tdist

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import system as S

    rank, world, local = dist_env()
    if world > 1:
        tdist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev_name = "cuda:%d" % local
    w, pos, mass = workload(args, rank)
    tune, tune_src = pick_tune(w, args)
    t0 = time.perf_counter()
    tree = S.Tree(pos, mass, w["leaf_size"])
    t1 = time.perf_counter()
    lists = tree.lists(w["theta"], w["n_crit"], w["eps"], w["use_quad"])
    t2 = time.perf_counter()
    plan = lists.plan(tune)
    t3 = time.perf_counter()
    dev = S.DeviceSystem.upload(lists, plan, dev_name)
    n = lists.n_part
    accel = torch.empty((n, 3), dtype=torch.float64, device=dev_name)
    pot = torch.empty(n, dtype=torch.float64, device=dev_name)
    stream = torch.cuda.current_stream()

    def step(prec):
        S.force(dev, accel, pot, precision=prec, tune=tune, stream=stream, check=False)

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        L.call("otoo_check_status", __import__("ctypes").byref(dev.struct), __import__("ctypes").c_void_p(stream.cuda_stream))
        if world > 1:
            tdist.barrier()
        torch.cuda.synchronize()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        evs[0].record(stream)
        for k in range(steps):
            step(prec)
            evs[k + 1].record(stream)
        torch.cuda.synchronize()
        per = [evs[k].elapsed_time(evs[k + 1]) for k in range(steps)]
        total = evs[0].elapsed_time(evs[-1])
        if world > 1:
            total = max_over_ranks(total, dev_name)
            tdist.barrier()
        return total, per

    with Clocks(local) as clk:
        total_ms, per_ms = timed(L.OTOO_FP32K, args.steps, args.warmup)
    clocks = clk.summary()
    a32 = accel.double().cpu().numpy()
    p32 = pot.double().cpu().numpy()
    inter = lists.interactions
    cell_inter = lists.cell_interactions if lists.use_quad else 0
    mono_inter = inter - cell_inter
    ms = total_ms / args.steps
    value = whole_job_rate(inter, world, ms)

    # FP64 form (the comparison form), same lists and launch shape
    fp64 = None
    if not args.skip_fp64:
        k64 = max(1, min(3, args.steps))
        tot64, _ = timed(L.OTOO_FP64, k64, 1)
        a64 = accel.double().cpu().numpy()
        p64 = pot.double().cpu().numpy()
        fp64 = {"value": inter / (tot64 / k64 * 1e-3), "ms_per_step": tot64 / k64,
                "fp32_vs_fp64_acc_max_rel": rel_err(a32, a64)[1]}

    # accuracy against the FP64 direct sum on a seeded subsample
    errors = None
    if rank == 0 and args.err_targets > 0:
        from paper_1206_1199_gb300 import ic
        sub = ic.subsample(n, args.err_targets, 7)
        # the library's FP64 direct sum on the device (checked against the oracle in the tests)
        ad, pd = S.direct_sum(pos, mass, w["eps"], sub, dev_name)
        rms, mx = rel_err(a32[sub], ad)
        errors = {"targets": int(sub.shape[0]), "fp32k_acc_rms": rms, "fp32k_acc_max": mx,
                  "fp32k_pot_rms": float(np.sqrt(np.mean(((p32[sub] - pd) / pd) ** 2)))}
        if fp64 is not None:
            rms64, mx64 = rel_err(a64[sub], ad)
            errors.update({"fp64_acc_rms": rms64, "fp64_acc_max": mx64})

    # end to end through the C ABI from pinned host buffers: the user's time
    # step (positions in, tree, walk, plan and force on the device,
    # accelerations out) and the force step on lists built by the host
    # (groups, lists and work items copied in)
    e2e = e2e_lists = step = None
    if not args.skip_step:
        step = guarded_extra(run_device_step, args, dev_name, pos, mass, w, tune, tree, lists, a32, stream, t1 - t0,
                             world)
    if not args.skip_e2e:
        e2e_lists = run_e2e(args, lists, plan, tune, stream, world)
    if step is not None and "error" not in step:
        e2e = {"value": step["value"], "unit": "interactions/s", "ms_per_step": step["step_wall_ms"],
               "h2d_bytes_per_step": step["h2d_bytes_per_step"], "d2h_bytes_per_step": step["d2h_bytes_per_step"],
               "steps": step["steps"],
               "path": "pinned host positions and masses copied in; tree, walk, plan and force on the device; "
                       "accelerations and potentials written by the force kernel into pinned host memory "
                       "(interactions equal to the host walk's)"}
    elif e2e_lists is not None:
        e2e = dict(e2e_lists, path="host-built groups, lists and work items copied in; force; results out")

    flops = 20.0 * mono_inter + (60.0 if lists.use_quad else 20.0) * cell_inter
    # the FP32 operations the pair kernels issue (fma = 2 flop; the MUFU
    # reciprocal square root not counted): 19 per particle or monopole pair,
    # 53 per quadrupole pair
    flops_code = 19.0 * mono_inter + (53.0 if lists.use_quad else 19.0) * cell_inter
    props = torch.cuda.get_device_properties(local)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (ms * 1e-3) / 1e12
    achieved_code = flops_code / (ms * 1e-3) / 1e12
    probe = guarded_extra(fma_probe, dev_name, local, stream) if rank == 0 else None
    measured = probe.get("tflops") if probe and "error" not in probe else None
    line = {
        "metric": "force interactions/s (FP32 centre-relative + Kahan) at N=2^23",
        "value": value,
        "unit": "interactions/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms,
        "ms_per_step_min": min(per_ms),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "model": w["model"], "n": n, "eps": w["eps"], "theta": w["theta"],
                   "leaf_size": w["leaf_size"], "n_crit": w["n_crit"], "quadrupole": bool(lists.use_quad),
                   "groups": lists.n_groups, "list_entries": lists.n_list, "interactions": inter,
                   "cell_interactions": cell_inter, "tune": tune.as_dict(), "tune_source": tune_src,
                   "items": plan.n_items, "list_length": list_length_stats(lists),
                   "l2": "inputs larger than L2 (%.1f GB resident per step)" % (dev.h2d_bytes() / 1e9),
                   "host_tree_s": t1 - t0, "host_walk_s": t2 - t1, "host_plan_s": t3 - t2,
                   "parallelism": "replica per rank (weak)"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": CAPTURED_TRAFFIC.get((args.workload, n, w["n_crit"],
                                                      (tune.block, tune.iblock, tune.tile, tune.split, tune.packed))),
                     "traffic_note": "DRAM bytes per force-kernel launch from one ncu capture of this configuration",
                     "timing": "achieved uses the CUDA-event time of the whole step (float-pair split 0.26 ms included)",
                     "flops_per_step": flops,
                     "peak_basis": "%d SMs x %d FP32 lanes x 2 flop x %.0f MHz max SM clock (derived from unit "
                                   "counts and the clock)" % (props.multi_processor_count, FP32_LANES_PER_SM, sm_max),
                     "flop_convention": "20 per monopole/particle interaction, 60 per quadrupole cell interaction",
                     "peak_measured": measured,
                     "frac_of_measured": achieved / measured if measured else None,
                     "fma_probe": probe,
                     "flops_code_per_step": flops_code,
                     "frac_code_flops": achieved_code / peak,
                     "code_flop_convention": "FP32 operations the pair kernels issue: 19 per particle/monopole pair, "
                                             "53 per quadrupole pair (fma = 2), reciprocal square root not counted"},
        "fp64_form": fp64,
        "errors": errors,
        "e2e": e2e,
        "e2e_host_lists": e2e_lists,
        "clocks": clocks,
        # per FP32 step: the float-pair split, the force kernel, the chunk merge when lists are split
        "gpu_launches": args.steps * (2 + (1 if plan.n_splits else 0)),
    }
    if rank == 0 and not args.skip_walk:
        line["device_walk"] = guarded_extra(run_device_walk, args, dev_name, tree, w, tune, lists, a32, stream,
                                            t2 - t1, t3 - t2)
    if rank == 0 and step is not None:
        line["device_step"] = step
    if rank == 0 and not args.skip_sph:
        line["sph_density"] = guarded_extra(run_sph, args, dev_name, pos, mass, w, stream)
    if rank == 0 and not args.skip_sw and errors is not None:
        line["sw_sweep"] = guarded_extra(run_sw_sweep, args, dev_name, tree, w, tune, stream, sub, ad)
    if rank == 0 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(w, pos, mass, args.cpu_fraction, args.cpu_repeats,
                                            direct=(sub[:128], ad[:128]) if errors is not None else None)
    if rank == 0 and not args.skip_extras and args.workload == "hernquist8m":
        line["fused_walk_force"] = guarded_extra(run_fused, args, dev_name, pos, mass, w, tune, stream)
        line["paper_workloads"] = guarded_extra(run_paper_workloads, args, dev_name, tune, stream)
        line["batch64"] = guarded_extra(run_batch, args, dev_name)
        line["learned_merger4m"] = guarded_extra(run_learned, args, dev_name)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()


def fma_probe(dev_name, local, stream):
    """Arithmetic throughput of this GPU (otoo_fma_probe: dependent chains of
    scalar fma.rn.f32 and packed fma.rn.f32x2 on every resident thread, the
    FP32 peak; fma.rn.f64 and rsqrt.approx.f32 for the rates the design
    weighs against it), CUDA events around 5 launches after one warm-up,
    clocks sampled.  Rates in T flop/s (T operations/s for rsqrt)."""
    import ctypes

    import torch

    from paper_1206_1199_gb300 import _lib as L
    n = int(L.load().otoo_fma_probe_threads())
    sink = torch.empty(max(n, 1), dtype=torch.float32, device=dev_name)
    out = {}
    st = ctypes.c_void_p(stream.cuda_stream)
    with Clocks(local) as clk:
        for kind, iters, key in ((0, 1 << 17, "fma_f32"), (1, 1 << 16, "fma_f32x2"), (2, 1 << 11, "fma_f64"),
                                 (3, 1 << 14, "rsqrt_f32")):
            fl = ctypes.c_double(0.0)
            L.call("otoo_fma_probe", iters, kind, sink.data_ptr(), ctypes.byref(fl), st)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(5):
                L.call("otoo_fma_probe", iters, kind, sink.data_ptr(), ctypes.byref(fl), st)
            e1.record(stream)
            torch.cuda.synchronize()
            out[key] = 5 * fl.value / (e0.elapsed_time(e1) * 1e-3) / 1e12
    c = clk.summary()
    mhz = c.get("sm_mhz") or c.get("sm_max_mhz")
    out["tflops"] = max(out["fma_f32"], out["fma_f32x2"])
    out["clocks"] = c
    if mhz:
        props = torch.cuda.get_device_properties(local)
        # FP32 flop per SM per clock at the sampled clock (128 lanes x 2 = 256 nominal)
        out["flop_per_sm_per_clock"] = out["tflops"] * 1e12 / (props.multi_processor_count * mhz * 1e6)
    return out


def guarded_extra(fn, *a):
    """An extra measurement must not cost the headline line."""
    try:
        return fn(*a)
    except Exception as e:  # reported in the JSON line
        return {"error": "%s: %s" % (type(e).__name__, e)}


def list_length_stats(lists):
    """Distribution of the groups' list lengths (cell + particle entries):
    quantiles and a histogram in powers of two (bin k: lengths in [2^k,
    2^(k+1)))."""
    g = lists.groups
    ln = (g["n_cell"].astype(np.int64) + g["n_part"].astype(np.int64))
    if len(ln) == 0:
        return {}
    q = np.quantile(ln, [0.0, 0.01, 0.5, 0.99, 1.0])
    k = np.floor(np.log2(np.maximum(ln, 1))).astype(int)
    hist = {str(1 << int(b)): int(c) for b, c in zip(*np.unique(k, return_counts=True))}
    return {"min": int(q[0]), "p01": float(q[1]), "median": float(q[2]), "p99": float(q[3]), "max": int(q[4]),
            "mean_cell_fraction": float(g["n_cell"].sum() / max(ln.sum(), 1)), "hist_log2": hist}


def run_device_walk(args, dev_name, tree, w, tune, lists, a32, stream, host_walk_s, host_plan_s):
    """The step with the walk and the plan on the device: otoo_walk_count,
    (host reads the list length), otoo_walk_fill, otoo_plan_count, (host
    reads the item count), otoo_plan_fill, otoo_force; buffers reused between
    steps.  Checked against the host walk's lists at full size (per-group
    entry counts, totals) and the FP32 forces on the host lists."""
    import torch

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import system as S
    t0 = time.perf_counter()
    dt = S.DeviceTree(tree, w["n_crit"], w["use_quad"], dev_name)
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t0
    pool = S.BufferPool(dev_name)
    n = lists.n_part
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev_name)
    pot = torch.empty(n, dtype=torch.float64, device=dev_name)

    def one():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        dl = dt.walk(w["theta"], w["eps"], stream=stream, pool=pool, group_set=args.walk_group_set)
        ev[1].record(stream)
        dp = dl.plan(tune, stream=stream)
        ev[2].record(stream)
        S.force(S.DeviceStep(dl, dp), acc, pot, L.OTOO_FP32K, tune, stream=stream, check=False)
        ev[3].record(stream)
        return dl, dp, ev

    for _ in range(2):
        one()
    torch.cuda.synchronize()
    times = []
    k = max(3, min(args.steps, 10))
    tw = time.perf_counter()
    for _ in range(k):
        dl, dp, ev = one()
        torch.cuda.synchronize()
        times.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]), ev[2].elapsed_time(ev[3])])
    wall = (time.perf_counter() - tw) / k
    med = np.median(np.array(times), axis=0)
    g, hg = dl.groups, lists.groups
    # entry counts per group (the offsets depend on the layout: slots of the one-pass walk)
    same = bool(np.array_equal(g["n_cell"], hg["n_cell"]) and np.array_equal(g["n_part"], hg["n_part"]))
    rms, mx = rel_err(acc.cpu().numpy(), a32)
    return {"walk_ms": float(med[0]), "plan_ms": float(med[1]), "force_ms": float(med[2]),
            "step_ms": float(med.sum()), "step_wall_ms": wall * 1e3, "steps": k,
            "host_walk_ms": host_walk_s * 1e3, "host_plan_ms": host_plan_s * 1e3,
            "walk_speedup_vs_host": host_walk_s * 1e3 / float(med[0]),
            "tree_arrays_s": prep_s, "tree_arrays_bytes": int(dt.h2d_bytes()),
            "group_counts_equal_host": same, "n_list": int(dl.n_list),
            "interactions_equal_host": bool(dl.interactions == lists.interactions),
            "items": int(dp.n_items), "fp32_vs_host_lists_acc_rms": rms, "fp32_vs_host_lists_acc_max": mx}


def run_device_step(args, dev_name, pos, mass, w, tune, tree, lists, a32, stream, host_tree_s, world=1):
    """The whole step on the device, from host positions to host
    accelerations: copy positions and masses in (pinned memory), build the
    tree (otoo_devtree_build), walk, plan, force; the force kernel writes
    the accelerations and potentials straight into pinned host memory
    (device-mapped), so their transfer to the host overlaps the kernel
    instead of following it as a copy.  Timed per step by the host clock
    (the tree build and the walk read a few sizes back, and the step ends
    when the outputs are in host memory); CUDA events split the device time.
    Checked against the host build: cell count, groups, per-group entry
    counts, FP32 accelerations."""
    import torch

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import system as S
    n = len(pos)
    pos_h = torch.from_numpy(np.ascontiguousarray(pos, np.float64)).pin_memory()
    mass_h = torch.from_numpy(np.ascontiguousarray(mass, np.float32)).pin_memory()
    pos_d = torch.empty_like(pos_h, device=dev_name)
    mass_d = torch.empty_like(mass_h, device=dev_name)
    # outputs: pinned host memory, written by the force kernel itself
    acc_h = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    pot_h = torch.empty(n, dtype=torch.float64).pin_memory()
    pool = S.BufferPool(dev_name)
    cap = [max(1024, n // 2)]

    def one():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        ev[0].record(stream)
        pos_d.copy_(pos_h, non_blocking=True)
        mass_d.copy_(mass_h, non_blocking=True)
        ev[1].record(stream)
        dt = S.DeviceTree.build(pos_d, mass_d, w["leaf_size"], w["n_crit"], w["use_quad"], dev_name,
                                cap_cell=cap[0], stream=stream)
        cap[0] = max(cap[0], dt.n_cell)
        ev[2].record(stream)
        dl = dt.walk(w["theta"], w["eps"], stream=stream, pool=pool, group_set=args.walk_group_set)
        ev[3].record(stream)
        dp = dl.plan(tune, stream=stream)
        S.force(S.DeviceStep(dl, dp), acc_h, pot_h, L.OTOO_FP32K, tune, stream=stream, check=False)
        ev[4].record(stream)
        torch.cuda.synchronize()
        return dt, dl, ev

    for _ in range(2):
        one()
    k = max(3, min(args.steps, 8))
    times, walls = [], []
    for _ in range(k):
        t0 = time.perf_counter()
        dt, dl, ev = one()
        walls.append(time.perf_counter() - t0)
        times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(4)])
    med = np.median(np.array(times), axis=0)
    wall = max_over_ranks(float(np.median(walls)), dev_name)  # the slowest rank's step
    hg, gd = lists.groups, dl.groups
    same_groups = bool(np.array_equal(gd["first"], hg["first"]) and np.array_equal(gd["count"], hg["count"]))
    same_counts = float(np.mean((gd["n_cell"] == hg["n_cell"]) & (gd["n_part"] == hg["n_part"])))
    rms, mx = rel_err(acc_h.numpy(), a32)
    return {"step_wall_ms": wall * 1e3, "steps": k, "h2d_ms": float(med[0]), "tree_ms": float(med[1]),
            "walk_ms": float(med[2]), "plan_force_ms": float(med[3]),
            "outputs": "written by the force kernel into pinned host memory (no separate copy)",
            "value": world * dl.interactions / wall, "unit": "interactions/s",
            "h2d_bytes_per_step": int(n * 28), "d2h_bytes_per_step": int(n * 32),
            "host_tree_ms": host_tree_s * 1e3, "n_cell": int(dt.n_cell),
            "n_cell_equal_host": bool(dt.n_cell == tree.export()["n_cell"]), "groups_equal_host": same_groups,
            "group_counts_equal_fraction": same_counts, "interactions": int(dl.interactions),
            "fp32_vs_host_path_acc_rms": rms, "fp32_vs_host_path_acc_max": mx}


def run_sph(args, dev_name, pos, mass, w, stream):
    """The SPH density stage (Section II, Eq. SPH_SUM, Eq. SPH_RAD) on the
    same particles, all on the device from device-resident positions: tree
    with r_SPH records, SPH walk, plan, density kernel; neighbour radii
    enclosing about 64 particles at the model's analytic density.  Checked
    against the FP64 direct sum on 256 targets."""
    import torch

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import ic
    from paper_1206_1199_gb300 import system as S
    h = ic.sph_radii(pos, mass, 64, w["model"])
    n = len(pos)
    tune = L.default_tune(w["n_crit"])
    tune.iblock = 2   # measured fastest for the density kernel (n_crit 128: 3.09 ms against 3.25 / 3.40 ms at 1 / 4)
    rho = torch.empty(n, dtype=torch.float64, device=dev_name)
    h_d = torch.from_numpy(h).to(dev_name)
    pos_d = torch.from_numpy(np.ascontiguousarray(pos, np.float64)).to(dev_name)
    mass_d = torch.from_numpy(np.ascontiguousarray(mass, np.float32)).to(dev_name)
    pool = S.BufferPool(dev_name)  # steady state of a time loop: the walk is one pass after the first step

    def one():
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        dt = S.DeviceTree.build(pos_d, mass_d, w["leaf_size"], w["n_crit"], False, dev_name, mac="sph", h_sph=h_d,
                                cap_cell=n // 2, stream=stream)
        ev[1].record(stream)
        dl = dt.walk(0.0, 1.0, stream=stream, pool=pool, group_set=args.walk_group_set)
        ev[2].record(stream)
        S.sph_density(S.DeviceStep(dl, dl.plan(tune, stream=stream)), h_d, rho, tune, stream=stream)
        ev[3].record(stream)
        torch.cuda.synchronize()
        return dl, ev

    one()
    times = []
    for _ in range(3):
        dl, ev = one()
        times.append([ev[i].elapsed_time(ev[i + 1]) for i in range(3)])
    med = np.median(np.array(times), axis=0)
    sub = ic.subsample(n, 256, 17)
    ref = S.sph_direct(pos, mass, h, sub, dev_name)  # FP64 brute force on the device, checked in the tests
    err = np.abs(rho.cpu().numpy()[sub] - ref) / ref
    return {"tree_ms": float(med[0]), "walk_ms": float(med[1]), "walk_one_pass": bool(dl.one_pass),
            "plan_density_ms": float(med[2]),
            "pairs": int(dl.interactions), "pairs_per_s": dl.interactions / (med[2] * 1e-3),
            "mean_list": dl.interactions / n, "n_ngb": 64, "targets": 256, "rel_err_max": float(err.max()),
            "rel_err_rms": float(np.sqrt(np.mean(err * err)))}


def run_sw_sweep(args, dev_name, tree, w, tune, stream, sub, ad):
    """The paper's accuracy control (Section II-B, Eq. SW_MAC): the absolute
    MAC over a range of delta with m_limit = 0.05 of the total mass, walked
    on the device; per delta the list size, the FP32 force-step time and the
    error against the FP64 direct sum on the error targets, and the slope of
    the cost against delta (the paper's model: delta^-3/4 for small delta)."""
    import torch

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import system as S
    m_limit = 0.05 * float(tree.export()["mass"].astype(np.float64).sum())
    rows = []
    n = tree.n
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev_name)
    pot = torch.empty(n, dtype=torch.float64, device=dev_name)
    for delta in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5):
        dt = S.DeviceTree(tree, w["n_crit"], w["use_quad"], dev_name, mac="sw", delta=delta, m_limit=m_limit)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        try:
            dl = dt.walk(0.0, w["eps"], stream=stream, max_entries=int(2.5e9), group_set=args.walk_group_set)
        except ValueError as e:
            rows.append({"delta": delta, "skipped": str(e)})
            break
        e1.record(stream)
        step = S.DeviceStep(dl, dl.plan(tune, stream=stream))
        S.force(step, acc, pot, L.OTOO_FP32K, tune, stream=stream)
        torch.cuda.synchronize()
        walk_ms = e0.elapsed_time(e1)
        k = 3
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        for _ in range(k):
            S.force(step, acc, pot, L.OTOO_FP32K, tune, stream=stream, check=False)
        f1.record(stream)
        torch.cuda.synchronize()
        ms = f0.elapsed_time(f1) / k
        rms, mx = rel_err(acc.cpu().numpy()[sub], ad)
        rows.append({"delta": delta, "interactions": int(dl.interactions), "cell_interactions":
                     int(dl.cell_interactions), "force_ms": ms, "walk_ms": walk_ms, "acc_rms": rms, "acc_max": mx})
        del step, dl, dt
        torch.cuda.empty_cache()
        if ms > 2000:
            break
    done = [r for r in rows if "interactions" in r]
    slopes = [math.log(b["interactions"] / a["interactions"]) / math.log(b["delta"] / a["delta"])
              for a, b in zip(done, done[1:])]
    return {"m_limit": m_limit, "rows": rows, "cost_slopes": slopes, "error_targets": int(len(sub))}


def run_fused(args, dev_name, pos, mass, w, tune, stream):
    """The walk fused with the force (otoo_walk_force: one warp per group
    walks and evaluates, no list in memory) against the split device step
    (one-pass walk into lists, plan, packed force) on the same device tree,
    for n_crit 64 (2 targets per lane) and 128 (4 per lane); errors against
    the FP64 direct sum on 256 targets."""
    import torch

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import ic
    from paper_1206_1199_gb300 import system as S
    n = len(pos)
    pos_d = torch.from_numpy(np.ascontiguousarray(pos)).to(dev_name)
    mass_d = torch.from_numpy(np.ascontiguousarray(mass)).to(dev_name)
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev_name)
    pot = torch.empty(n, dtype=torch.float64, device=dev_name)
    sub = ic.subsample(n, 256, 13)
    ad, _ = S.direct_sum(pos, mass, w["eps"], sub, dev_name)
    rows = []

    def timed(fn, k=5):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    for nc, ib in ((64, 2), (128, 4)):
        dt = S.DeviceTree.build(pos_d, mass_d, w["leaf_size"], nc, w["use_quad"], dev_name, stream=stream)
        fs = dt.fused(w["theta"], w["eps"], ib)
        fused_ms = timed(lambda: fs(acc, pot, stream=stream, check=False))
        fs(acc, pot, stream=stream)
        rms, mx = rel_err(acc.cpu().numpy()[sub], ad)
        nl, inter, cinter = fs.totals()
        t = L.Tune(block=128, iblock=2, tile=256, split=8192, ctas_per_sm=0, packed=1)
        pool = S.BufferPool(dev_name)
        dt.walk(w["theta"], w["eps"], stream=stream, pool=pool, group_set=args.walk_group_set)

        def split_step():
            dl = dt.walk(w["theta"], w["eps"], stream=stream, pool=pool, group_set=args.walk_group_set)
            S.force(S.DeviceStep(dl, dl.plan(t, stream=stream)), acc, pot, L.OTOO_FP32K, t, stream=stream,
                    check=False)

        split_ms = timed(split_step)
        rows.append({"n_crit": nc, "iblock": ib, "interactions": int(inter), "cell_interactions": int(cinter),
                     "fused_ms": fused_ms, "split_walk_plan_force_ms": split_ms,
                     "fused_interactions_per_s": inter / (fused_ms * 1e-3), "acc_rms": rms, "acc_max": mx})
        del dt, fs, pool
        torch.cuda.empty_cache()
    return {"rows": rows, "error_targets": 256}


# The paper's own gravity benchmark (Section IV-A): N = 8M Plummer model and
# uniform sphere, absolute MAC with delta = 0.01 and m_limit = 0.05, monopole
# cells, tree leaves of 16; its OpenCL kernel time per step on one Tesla
# M2090 (walk and force fused on the GPU, single precision).
PAPER_WORKLOADS = (("plummer", 1 << 23, 2.08, "1x Tesla M2090 (2012), OpenCL, walk and force fused"),
                   ("uniform", 8000 * 1024, 1.52, "1x Tesla M2090 (2012), OpenCL, walk and force fused"))


def run_paper_workloads(args, dev_name, tune, stream):
    """The paper's gravity benchmark configurations, for context beside its
    published kernel times: device tree (leaf size 16), device walk with the
    absolute MAC (delta 0.01, m_limit 0.05), plan and FP32 force (monopole
    cells, eps 1e-3: the paper gives no softening); errors against the FP64
    direct sum on 256 targets.  On the uniform sphere also the delta sweep of
    the paper's Figs. 4 and 5 (walk + force time and mean error against
    delta, their slopes between successive deltas)."""
    import torch

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import ic
    from paper_1206_1199_gb300 import system as S
    out = []
    eps = 1e-3

    def measure(pos_d, mass_d, n, delta, sub, ad):
        acc = torch.empty((n, 3), dtype=torch.float64, device=dev_name)
        pot = torch.empty(n, dtype=torch.float64, device=dev_name)

        def one():
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            dt = S.DeviceTree.build(pos_d, mass_d, 16, 128, False, dev_name, mac="sw", delta=delta, m_limit=0.05,
                                    stream=stream)
            ev[1].record(stream)
            dl = dt.walk(0.0, eps, stream=stream, group_set=args.walk_group_set)
            ev[2].record(stream)
            S.force(S.DeviceStep(dl, dl.plan(tune, stream=stream)), acc, pot, L.OTOO_FP32K, tune, stream=stream)
            ev[3].record(stream)
            torch.cuda.synchronize()
            return dl, [ev[i].elapsed_time(ev[i + 1]) for i in range(3)]

        one()
        runs = [one() for _ in range(3)]
        dl = runs[-1][0]
        med = np.median(np.array([r[1] for r in runs]), axis=0)
        d = np.linalg.norm(acc.cpu().numpy()[sub] - ad, axis=1) / np.linalg.norm(ad, axis=1)
        row = {"delta": delta, "interactions": int(dl.interactions), "tree_ms": float(med[0]),
               "walk_ms": float(med[1]), "plan_force_ms": float(med[2]), "gravity_ms": float(med[1] + med[2]),
               "acc_mean": float(d.mean()), "acc_rms": float(np.sqrt(np.mean(d * d))), "acc_max": float(d.max())}
        del dl, runs, acc, pot
        torch.cuda.empty_cache()
        return row

    sweep = None
    for model, n, paper_s, paper_hw in PAPER_WORKLOADS:
        pos, mass = ic.make(model, n, ic.BASE_SEED + 6)
        pos_d = torch.from_numpy(np.ascontiguousarray(pos)).to(dev_name)
        mass_d = torch.from_numpy(np.ascontiguousarray(mass)).to(dev_name)
        sub = ic.subsample(n, 256, 11)
        ad, _ = S.direct_sum(pos, mass, eps, sub, dev_name)
        row = measure(pos_d, mass_d, n, 0.01, sub, ad)
        row.update(model=model, n=n, error_targets=256, paper_kernel_s=paper_s, paper_hardware=paper_hw)
        out.append(row)
        if model == "uniform":
            rows = [measure(pos_d, mass_d, n, dlt, sub, ad) for dlt in (1e-1, 3e-2, 1e-2, 3e-3, 1e-3)]
            lg = lambda a, b, k: math.log(b[k] / a[k]) / math.log(b["delta"] / a["delta"])  # noqa: E731
            sweep = {"rows": rows,
                     "time_slopes": [lg(a, b, "gravity_ms") for a, b in zip(rows, rows[1:])],
                     "mean_error_slopes": [lg(a, b, "acc_mean") for a, b in zip(rows, rows[1:])],
                     "paper": "time ~ delta^-3/4 (Section II-B, Fig. 4); mean error ~ delta^0.25 at small delta "
                              "(Fig. 5)"}
        del pos_d, mass_d
        torch.cuda.empty_cache()
    return {"mac": "absolute, delta 0.01, m_limit 0.05", "cells": "monopole", "leaf_size": 16, "n_crit": 128,
            "eps": eps, "rows": out, "uniform_delta_sweep": sweep}


def run_batch(args, dev_name):
    """64 independent Plummer/King systems of uneven size packed into one
    ragged buffer and evaluated by one graph-launched force step."""
    import torch

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import ic
    from paper_1206_1199_gb300 import system as S
    w = ic.WORKLOADS["batch64"]
    systems = ic.batch_systems(w["n_sys"], w["seed"])
    t0 = time.perf_counter()
    per = [S.Tree(p, m, w["leaf_size"]).lists(w["theta"], w["n_crit"], e, w["use_quad"]) for p, m, e in systems]
    packed = S.Lists.pack(per)
    host_s = time.perf_counter() - t0
    # the packed kernel with 256-entry tiles, as the autotuner picks for N = 2^23
    tune = L.Tune(block=128, iblock=2, tile=256, split=16384, ctas_per_sm=0, packed=1)
    dev = S.DeviceSystem.upload(packed, packed.plan(tune), dev_name)
    n = packed.n_part
    acc = torch.empty((n, 3), dtype=torch.float64, device=dev_name)
    pot = torch.empty(n, dtype=torch.float64, device=dev_name)
    for _ in range(3):
        S.force(dev, acc, pot, L.OTOO_FP32K, tune)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        S.force(dev, acc, pot, L.OTOO_FP32K, tune, check=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    a = acc.cpu().numpy()
    S.force(dev, acc, pot, L.OTOO_FP64, tune)
    a64 = acc.cpu().numpy()
    # every system against its own FP64 direct sum on the device, min(N, 1024) targets
    from paper_1206_1199_gb300.learned import Evaluator
    rms32, rms64 = [], []
    off = packed.sys_part_off
    for k, (p, m, e) in enumerate(systems):
        ev = Evaluator(p, m, e, w["n_crit"], device=dev_name)
        sub = ic.subsample(len(p), 1024, 300 + k)
        perm = ev.tree.export()["perm"]
        inv = np.empty_like(perm)
        inv[perm] = np.arange(len(perm))
        ad, _ = ev.direct(inv[sub])
        rms32.append(rel_err(a[off[k] + sub], ad)[0])
        rms64.append(rel_err(a64[off[k] + sub], ad)[0])
    worst = int(np.argmax(rms32))
    return {"systems": len(systems), "n_total": int(n), "interactions": int(packed.interactions),
            "ms_per_step": ms, "value": packed.interactions / (ms * 1e-3), "unit": "interactions/s",
            "host_tree_walk_s": host_s, "worst_system": worst, "worst_system_n": len(systems[worst][0]),
            "worst_system_acc_rms": rms32[worst], "worst_system_acc_rms_fp64_form": rms64[worst],
            "median_system_acc_rms": float(np.median(rms32)), "error_targets_per_system": "min(N, 1024)"}


def run_learned(args, dev_name):
    """Learned per-group angles (network trained on method-generated
    snapshots of the two-polytrope system) against the fixed angle with the
    same RMS error, on an independent realisation of that system."""
    from paper_1206_1199_gb300 import ic, learned
    from paper_1206_1199_gb300.mlp import ThetaNet
    wpath = os.path.join(ROOT, "paper_1206_1199_gb300", "thetanet_merger4m.npz")
    if not os.path.exists(wpath):
        return {"error": "no trained network file"}
    w = ic.WORKLOADS["merger4m"]
    net = ThetaNet.load(wpath, dev_name)
    pos, mass, _ = learned.merger_ic(w["n"], w["seed"] + 100)
    ev = learned.Evaluator(pos, mass, w["eps"], w["n_crit"], device=dev_name)
    res = learned.compare(ev, net, 1e-3, n_sub=2048, bisect_steps=7)
    res["n"] = w["n"]
    return res


def run_e2e(args, lists, plan, tune, stream, world):
    """Same metric through otoo_force_host: pinned host inputs copied in and
    results copied out inside the timed region, every step."""
    import ctypes

    import torch

    from paper_1206_1199_gb300 import _lib as L
    from paper_1206_1199_gb300 import system as S

    v = L.ListsView()
    ctypes.memmove(ctypes.byref(v), ctypes.byref(lists.view_struct), ctypes.sizeof(v))
    keep = []
    h2d = 0
    for field, arr in (("src", lists.src), ("quad", lists.quad), ("groups", lists.groups), ("list", lists.list),
                       ("perm", lists.perm)):
        t = torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).reshape(-1)).pin_memory()
        keep.append(t)
        setattr(v, field, t.data_ptr())
        if field != "quad" or lists.use_quad:
            h2d += t.numel()
    info = L.PlanInfo()
    ctypes.memmove(ctypes.byref(info), ctypes.byref(plan.info), ctypes.sizeof(info))
    for field, arr in (("items", plan.items), ("splits", plan.splits)):
        t = torch.from_numpy(np.ascontiguousarray(arr).view(np.uint8).reshape(-1).copy()
                             if arr.size else np.zeros(16, np.uint8)).pin_memory()
        keep.append(t)
        setattr(info, field, t.data_ptr())
        h2d += t.numel() if arr.size else 0
    n = lists.n_part
    acc = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    pot = torch.empty(n, dtype=torch.float64).pin_memory()
    d2h = (acc.numel() + pot.numel()) * 8
    steps = max(1, min(args.steps, 5))

    def one():
        L.call("otoo_force_host", ctypes.byref(v), ctypes.byref(info), acc.data_ptr(), pot.data_ptr(),
               L.OTOO_FP32K, ctypes.byref(tune), ctypes.c_void_p(stream.cuda_stream))

    one()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        one()
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    return {"value": world * lists.interactions / dt, "unit": "interactions/s", "ms_per_step": dt * 1e3,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h), "steps": steps}


def oracle_tree(w, pos, mass):
    import oracle
    return oracle.Tree(pos, mass, w["leaf_size"], w["n_crit"])


CPU_SAMPLE_SEED = 12061199 + 777  # the groups both arms time on the CPU


def cpu_sample(t, fraction):
    """A seeded random sample of the oracle tree's groups (the same groups in
    both arms and on every run of a workload)."""
    from paper_1206_1199_gb300 import ic
    k = max(1, min(t.n_groups, int(round(t.n_groups * fraction))))
    return ic.subsample(t.n_groups, k, CPU_SAMPLE_SEED)


def cpu_time_sample(w, t, sel):
    """(interactions, seconds) of the FP64 oracle tree force -- walk and
    evaluation of the sampled groups only -- on all host cores."""
    t0 = time.perf_counter()
    r = t.eval(w["theta"], w["eps"], w["use_quad"], groups=sel)
    return r["interactions"], time.perf_counter() - t0


def cpu_sample_text(t, sel, fraction, inter, secs):
    return ("FP64 oracle tree force (walk + evaluation) of a seeded random sample of %d of %d groups (fraction "
            "%.4g, seed %d): %d interactions, %.2f s per run; oracle tree build not timed"
            % (len(sel), t.n_groups, fraction, CPU_SAMPLE_SEED, inter, secs))


def cpu_baseline(w, pos, mass, fraction, repeats, tree=None, direct=None):
    """The FP64 oracle tree code (as it stands) on a seeded sample of the
    workload's groups, timed `repeats` times: median rate and its spread.
    direct = (targets, acc): also the oracle's FP64 direct sum on those
    targets, timed, and its largest relative difference from acc (the
    library's FP64 direct sum on the device, the reference of the line's
    errors)."""
    t = tree if tree is not None else oracle_tree(w, pos, mass)
    sel = cpu_sample(t, fraction)
    runs = [cpu_time_sample(w, t, sel) for _ in range(max(1, repeats))]
    rates = [i / max(s, 1e-9) for i, s in runs]
    med = float(np.median(rates))
    out = {"value": med, "unit": "interactions/s", "cores": cores(), "kind": "oracle", "repeats": len(runs),
           "spread": [float(min(rates)), float(max(rates))],
           "sample": cpu_sample_text(t, sel, fraction, runs[0][0], float(np.median([s for _, s in runs])))}
    if direct is not None:
        import oracle
        tgt, acc = direct
        t0 = time.perf_counter()
        ao, _ = oracle.direct(pos, mass, w["eps"], tgt)
        sec = time.perf_counter() - t0
        pairs = int(len(tgt)) * (len(pos) - 1)
        out["direct_sum"] = {"targets": int(len(tgt)), "pairs": pairs, "seconds": sec, "pairs_per_s": pairs / sec,
                             "library_fp64_direct_vs_oracle_max_rel": rel_err(acc, ao)[1]}
    return out


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    w, pos, mass = workload(args, 0)
    pick_tune(w, args)  # the same n_crit as the GPU arm
    tree = oracle_tree(w, pos, mass)
    sel = cpu_sample(tree, args.cpu_fraction)
    runs = []
    for k in range(args.warmup + args.steps):
        r = cpu_time_sample(w, tree, sel)
        if k >= args.warmup:
            runs.append(r)
    rates = [i / max(s, 1e-9) for i, s in runs]
    value = float(np.median(rates))
    # one whole step at the sample's rate: the sample's time scaled by the
    # fraction of the groups it holds
    ms_step = float(np.median([s for _, s in runs])) * 1e3 * tree.n_groups / max(len(sel), 1)
    line = {"impl": "reference", "metric": "force interactions/s (FP32 centre-relative + Kahan) at N=2^23",
            "value": value, "unit": "interactions/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step,
            "ms_per_step_note": "median sample time scaled to all groups (each step times a bounded sample)",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "model": w["model"], "n": w["n"], "eps": w["eps"],
                       "theta": w["theta"], "n_crit": w["n_crit"], "quadrupole": w["use_quad"]},
            "cpu_baseline": {"value": value, "unit": "interactions/s", "cores": cores(), "kind": "oracle",
                             "repeats": len(runs), "spread": [float(min(rates)), float(max(rates))],
                             "sample": cpu_sample_text(tree, sel, args.cpu_fraction, runs[-1][0],
                                                       float(np.median([s for _, s in runs])))},
            "e2e": {"value": value, "unit": "interactions/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def run_fused_only(args):
    """The fused walk + force comparison alone (rank 0, one JSON line)."""
    import torch
    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    w, pos, mass = workload(args, 0)
    tune, _ = pick_tune(w, args)
    r = run_fused(args, "cuda:%d" % local, pos, mass, w, tune, torch.cuda.current_stream())
    print(json.dumps({"workload": args.workload, "n": len(pos), "fused_walk_force": r}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.fused_only:
        run_fused_only(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
