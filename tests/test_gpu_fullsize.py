"""Parity at the full workload sizes, in the launch configuration the bench
times (autotuned n_crit and tune where cached), on sampled outputs the CPU
oracle can compute one by one:

* Hernquist N = 2^23, theta 0.5, quadrupole: FP32 form against the FP64
  direct sum on 256 sampled particles (RMS <= 2e-3); FP64 form against the
  oracle's tree force on every 2000th oracle group (<= 1e-6).
* Plummer N = 2^20, theta in {0.3, 0.5, 0.75}, n_crit 128, quadrupole: FP32
  form against the FP64 form on all particles (arithmetic only) and against
  the direct sum on 512 sampled particles."""
import numpy as np
import pytest

import oracle
from paper_1206_1199_gb300 import _lib as L
from paper_1206_1199_gb300 import autotune, ic, system as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


@pytest.fixture(scope="module")
def hernquist():
    import torch  # noqa: F401
    L.load()
    w = dict(ic.WORKLOADS["hernquist8m"])
    entry = autotune.lookup(w)
    if entry:
        w["n_crit"] = int(entry["n_crit"])
        tune = L.Tune(**{k: int(v) for k, v in entry["tune"].items()})
    else:
        tune = L.default_tune(w["n_crit"])
    pos, mass = ic.make(w["model"], w["n"], w["seed"])
    tree, lists, plan = S.build_system(pos, mass, w["theta"], w["n_crit"], w["eps"], w["leaf_size"], True, tune)
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    return w, pos, mass, lists, dev, tune


def test_fullsize_fp32_vs_direct_sum(hernquist):
    w, pos, mass, lists, dev, tune = hernquist
    a, p = S.force(dev, precision=L.OTOO_FP32K, tune=tune)
    a = a.cpu().numpy()
    sub = ic.subsample(w["n"], 256, 99)
    ad, pd = oracle.direct(pos, mass, w["eps"], targets=sub)
    d = rel(a[sub], ad)
    assert np.sqrt(np.mean(d * d)) <= 2e-3 and d.max() < 1e-2
    assert np.all(np.isfinite(a))


def test_fullsize_fp64_vs_oracle_tree(hernquist):
    w, pos, mass, lists, dev, tune = hernquist
    a, p = S.force(dev, precision=L.OTOO_FP64, tune=tune)
    a, p = a.cpu().numpy(), p.cpu().numpy()
    t = oracle.Tree(pos, mass, w["leaf_size"], w["n_crit"])
    r = t.eval(w["theta"], w["eps"], True, group_stride=2000)
    done = np.isfinite(r["pot"])
    assert done.sum() > 1000
    assert rel(a[done], r["acc"][done]).max() <= 1e-6
    assert (np.abs(p[done] - r["pot"][done]) / np.abs(r["pot"][done])).max() <= 1e-6


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.75])
def test_fullsize_plummer_theta_sweep(theta):
    import torch  # noqa: F401
    w = ic.WORKLOADS["plummer1m"]
    pos, mass = ic.make(w["model"], w["n"], w["seed"])
    tree, lists, plan = S.build_system(pos, mass, theta, w["n_crit"], w["eps"], w["leaf_size"], True)
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    a32, p32 = S.force(dev, precision=L.OTOO_FP32K)
    a64, p64 = S.force(dev, precision=L.OTOO_FP64)
    a32, a64 = a32.cpu().numpy(), a64.cpu().numpy()
    d = rel(a32, a64)
    assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4
    sub = ic.subsample(w["n"], 512, 98)
    ad, _ = oracle.direct(pos, mass, w["eps"], targets=sub)
    e = rel(a32[sub], ad)
    rms = np.sqrt(np.mean(e * e))
    if theta <= 0.5:
        assert rms <= 2e-3
    assert rms <= {0.3: 1e-4, 0.5: 5e-4, 0.75: 3e-3}[theta]


def test_fullsize_batch_of_64_systems():
    # 64 Plummer / King systems of 2^10..2^18 particles packed into one
    # ragged buffer and one launch in the bench's tune: every system's FP32
    # forces against its own FP64 direct sum (min(N, 1024) sampled targets,
    # RMS <= 2e-3 at theta 0.5), the FP64 form of the same launch beside it;
    # the packed launch bit-identical to separate launches (a spread of sizes)
    import torch  # noqa: F401
    L.load()
    w = ic.WORKLOADS["batch64"]
    systems = ic.batch_systems(w["n_sys"], w["seed"])
    sizes = np.array([len(p) for p, _, _ in systems])
    assert len(systems) == 64 and sizes.min() >= 2 ** 10 and sizes.max() <= 2 ** 18
    per = [S.Tree(p, m, w["leaf_size"]).lists(w["theta"], w["n_crit"], e, w["use_quad"]) for p, m, e in systems]
    packed = S.Lists.pack(per)
    tune = L.Tune(block=128, iblock=2, tile=256, split=16384, ctas_per_sm=0, packed=1)
    dev = S.DeviceSystem.upload(packed, packed.plan(tune), "cuda")
    a32, p32 = S.force(dev, precision=L.OTOO_FP32K, tune=tune)
    a64, _ = S.force(dev, precision=L.OTOO_FP64, tune=tune)
    a32, p32, a64 = a32.cpu().numpy(), p32.cpu().numpy(), a64.cpu().numpy()
    off = packed.sys_part_off
    rms32, rms64 = [], []
    for k, (pos, mass, eps) in enumerate(systems):
        sub = ic.subsample(len(pos), 1024, 300 + k)
        ad, _ = oracle.direct(pos, mass, eps, targets=sub)
        d32 = rel(a32[off[k] + sub], ad)
        d64 = rel(a64[off[k] + sub], ad)
        rms32.append(np.sqrt(np.mean(d32 * d32)))
        rms64.append(np.sqrt(np.mean(d64 * d64)))
    rms32, rms64 = np.array(rms32), np.array(rms64)
    worst = int(np.argmax(rms32))
    print("batch64: worst system %d (N = %d) FP32 RMS %.3e, FP64 form %.3e" % (worst, sizes[worst], rms32[worst],
                                                                              rms64[worst]))
    assert rms32.max() <= 2e-3
    # the FP32 form adds arithmetic error only to the tree error of theta
    assert np.all(np.abs(rms32 - rms64) <= 1e-5 + 1e-2 * rms64)
    order = np.argsort(sizes)
    for k in (int(order[0]), int(order[21]), int(order[42]), int(order[-1])):
        d = S.DeviceSystem.upload(per[k], per[k].plan(tune), "cuda")
        ak, pk = S.force(d, precision=L.OTOO_FP32K, tune=tune)
        np.testing.assert_array_equal(a32[off[k]:off[k + 1]], ak.cpu().numpy())
        np.testing.assert_array_equal(p32[off[k]:off[k + 1]], pk.cpu().numpy())
