"""Learned opening angle on the GPU: the device direct sum, the training
labels (group errors) and the selection against the FP64 CPU oracle, and
the gain of the trained network over a fixed angle at equal error."""
import numpy as np
import pytest

import oracle
from paper_1206_1199_gb300 import _lib as L
from paper_1206_1199_gb300 import ic
from paper_1206_1199_gb300 import system as S

pytestmark = pytest.mark.gpu

# interactions saved by the learned angles at equal RMS error on an
# independent realisation (1.108 measured with the committed network)
GAIN_MIN = 1.10


@pytest.fixture(scope="module")
def LR():
    import torch  # noqa: F401
    L.load()
    from paper_1206_1199_gb300 import learned
    return learned


def test_device_direct_sum_matches_oracle(LR):
    pos, mass = ic.plummer(5000, 41)
    ev = LR.Evaluator(pos, mass, 0.01)
    perm = ev.tree.export()["perm"]
    tgt = np.array([0, 1, 17, 2500, 4999])
    a, p = ev.direct(tgt)
    ar, pr = oracle.direct(pos, mass, 0.01, targets=perm[tgt])
    np.testing.assert_allclose(a, ar, rtol=0, atol=1e-12 * np.abs(ar).max())
    np.testing.assert_allclose(p, pr, rtol=1e-12)


def test_device_direct_sum_matches_oracle_at_a_million(LR):
    # the direct sum the bench's error figures use, at a size where it runs
    # in many source chunks (merged in order), against the oracle's
    pos, mass = ic.hernquist(1 << 20, 43)
    tgt = ic.subsample(1 << 20, 64, 44)
    a, p = S.direct_sum(pos, mass, 5e-4, tgt)
    ar, pr = oracle.direct(pos, mass, 5e-4, targets=tgt)
    assert np.all(np.linalg.norm(a - ar, axis=1) <= 1e-11 * np.linalg.norm(ar, axis=1))
    np.testing.assert_allclose(p, pr, rtol=1e-11)


def test_group_labels_match_oracle(LR):
    # the label of (group, angle) = RMS over the group's particles of the
    # relative force error of the tree force against the direct sum
    pos, mass = ic.polytrope_pair(20000, 42)
    eps = 1e-4
    ev = LR.Evaluator(pos, mass, eps, n_crit=64)
    grid = (0.3, 0.6, 0.9)
    X, y = LR.group_rows(ev, 40, grid=grid, theta0=0.5, seed=3)
    base = ev.lists(0.5)
    g = base.groups
    perm = base.perm
    rng = np.random.Generator(np.random.PCG64(3))
    sel = np.sort(rng.choice(base.n_groups, size=40, replace=False))
    keys = np.array([perm[g["first"][k]:g["first"][k] + g["count"][k]].min() for k in sel])
    ot = oracle.Tree(pos, mass, 8, 64)
    members = [perm[g["first"][k]:g["first"][k] + g["count"][k]] for k in sel]
    tg = np.concatenate(members)
    ad, _ = oracle.direct(pos, mass, eps, targets=tg)
    off = np.cumsum([0] + [len(m) for m in members])
    for a_i, th in enumerate(grid):
        tbk = np.full(len(pos), 0.5)
        tbk[keys] = th
        r = ot.eval(0.5, eps, True, theta_by_key=tbk)
        d = np.linalg.norm(r["acc"][tg] - ad, axis=1) / np.linalg.norm(ad, axis=1)
        rms = np.array([np.sqrt(np.mean(d[off[j]:off[j + 1]] ** 2)) for j in range(len(sel))])
        got = 10.0 ** y[a_i * len(sel):(a_i + 1) * len(sel)]
        np.testing.assert_allclose(got, rms, rtol=2e-2, atol=2e-6)
        np.testing.assert_array_equal(X[a_i * len(sel):(a_i + 1) * len(sel), 5], np.float32(th))


def test_training_pipeline_reaches_its_target(LR):
    # the whole pipeline on a small system: method-generated snapshots, rows,
    # training on the GPU, calibration on two training snapshots; on a later
    # snapshot the selection lands near its RMS target (the small system's
    # statistics are too noisy for a gain)
    pos, mass, vel = LR.merger_ic(1 << 16)
    eps = 4e-4
    dt = LR.orbital_period() / 200
    snaps = LR.leapfrog_snapshots(pos, mass, vel, eps, dt, 5, 2)
    X, y = LR.training_set(snaps[:4], mass, eps, groups_per_snap=128)
    net, hist = LR.train(X, y, steps=1500, batch=4096)
    assert hist[-1] < 0.5 * hist[0]
    LR.calibrate(net, [LR.Evaluator(snaps[k], mass, eps) for k in (0, 3)], 1e-3, iters=3)
    ev = LR.Evaluator(snaps[4], mass, eps)
    res = LR.compare(ev, net, target_rms=1e-3, n_sub=2048, precision_fp64=False, bisect_steps=6)
    assert 0.6e-3 < res["learned"]["rms"] < 1.4e-3, res["learned"]
    assert abs(res["fixed_equal_rms"]["rms"] - res["learned"]["rms"]) < 0.25 * res["learned"]["rms"]


def test_trained_network_on_an_independent_realisation(LR):
    # the committed network (trained on 16 method-generated snapshots of the
    # N = 2^22 two-polytrope system, calibrated on four of them) on another
    # realisation of that system: it meets its target, and at equal RMS it
    # needs fewer interactions than the fixed angle, with a p99 error no worse
    import os

    from paper_1206_1199_gb300 import ic
    from paper_1206_1199_gb300.mlp import ThetaNet
    path = os.path.join(os.path.dirname(LR.__file__), "thetanet_merger4m.npz")
    net = ThetaNet.load(path)
    w = ic.WORKLOADS["merger4m"]
    pos, mass, _ = LR.merger_ic(w["n"], w["seed"] + 100)
    ev = LR.Evaluator(pos, mass, w["eps"], w["n_crit"])
    res = LR.compare(ev, net, 1e-3, n_sub=4096, precision_fp64=False, bisect_steps=8)
    lr, fx = res["learned"], res["fixed_equal_rms"]
    print("learned angles on an independent realisation: RMS %.3e (fixed %.3e), gain %.3f interactions, %.3f time, "
          "p99 %.2e (fixed %.2e), max %.2e (fixed %.2e)" % (lr["rms"], fx["rms"], res["gain_interactions"],
                                                           res["gain_time"], lr["p99"], fx["p99"], lr["max"],
                                                           fx["max"]))
    assert 0.6e-3 <= lr["rms"] <= 1.1e-3, lr
    assert abs(fx["rms"] - lr["rms"]) < 0.1 * lr["rms"], (fx, lr)
    assert res["gain_interactions"] >= GAIN_MIN, res
    assert lr["p99"] <= fx["p99"], (lr, fx)


def test_direct_sum_helper_matches_oracle(LR):
    pos, mass = ic.plummer(5000, 12)
    tgt = ic.subsample(5000, 200, 3)
    a, p = S.direct_sum(pos, mass, 0.01, tgt)
    ar, pr = oracle.direct(pos, mass, 0.01, targets=tgt)
    np.testing.assert_allclose(a, ar, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p, pr, rtol=1e-12)


def test_snapshot_checkpoint_resumes_bit_for_bit(LR, tmp_path):
    # a snapshot run stopped after two snapshots, written to a checkpoint and
    # continued from it reaches the same third snapshot as the run that was
    # never stopped (the forces are deterministic)
    pos, mass, vel = LR.merger_ic(1 << 13)
    eps, dt = 1e-3, LR.orbital_period() / 200
    vels = []
    full = LR.leapfrog_snapshots(pos, mass, vel, eps, dt, 3, 2, velocities=vels)
    assert len(full) == len(vels) == 3
    part_v = []
    part = LR.leapfrog_snapshots(pos, mass, vel, eps, dt, 2, 2, velocities=part_v)
    path = str(tmp_path / "snaps.npz")
    LR.save_snapshots(path, part, part_v, mass, dt=dt, every=2, eps=eps)
    xs, vs, m, meta = LR.load_snapshots(path)
    assert meta == {"dt": dt, "every": 2, "eps": eps} and np.array_equal(m, mass)
    rest = LR.leapfrog_snapshots(None, mass, None, eps, dt, 3, 2, resume=(xs, vs, len(xs)))
    assert len(rest) == 3
    for a, b in zip(rest, full):
        np.testing.assert_array_equal(a, b)
