"""The walk fused with the FP32 force (otoo_walk_force, needs a GPU).

The fused kernel walks each group exactly as the device walk does and
evaluates the entries it finds with the packed FP32 pair arithmetic, so its
lists are the host walk's lists (same counts: totals equal) and its forces
differ from the FP64 form on those lists by FP32 rounding only: the
tolerance of the FP32 form against the FP64 form on identical lists (RMS <=
2e-6, max <= 2e-4 relative per particle), with the FP64 form itself pinned
to the FP64 oracle tree in test_gpu_force.py and test_gpu_walk.py."""
import ctypes

import numpy as np
import pytest

from paper_1206_1199_gb300 import _lib as L
from paper_1206_1199_gb300 import ic, system as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    L.load()
    return t


def lattice(k, scale=2.0, shift=10.0):
    g = (np.arange(k) + 0.5) / k
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * scale + shift
    return pos, np.full(len(pos), 1.0 / len(pos), np.float32)


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def fp64_on_host_lists(hl, ncrit):
    dev = S.DeviceSystem.upload(hl, hl.plan(L.default_tune(ncrit)), "cuda")
    return (x.cpu().numpy() for x in S.force(dev, precision=L.OTOO_FP64))


def run_fused(torch, fs, n):
    acc = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    pot = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    fs(acc, pot)
    return acc.cpu().numpy(), pot.cpu().numpy()


def check_fp32(a32, p32, a64, p64):
    d = rel(a32, a64)
    assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4, (np.sqrt(np.mean(d * d)), d.max())
    assert (np.abs(p32 - p64) / np.abs(p64)).max() <= 1e-5


@pytest.mark.parametrize("model,n,theta,ncrit,iblock,quad", [
    ("plummer", 20000, 0.5, 64, 2, True), ("hernquist", 30000, 0.75, 32, 1, True),
    ("plummer", 20000, 0.3, 128, 4, True), ("king", 8000, 0.6, 64, 2, False),
    ("lattice", 4096, 0.5, 64, 2, True)])
def test_fused_matches_fp64_form_on_host_lists(torch, model, n, theta, ncrit, iblock, quad):
    pos, mass = lattice(16) if model == "lattice" else ic.make(model, n, 61)
    n = len(pos)
    t = S.Tree(pos, mass, 8)
    hl = t.lists(theta, ncrit, 0.01, quad)
    a64, p64 = fp64_on_host_lists(hl, ncrit)
    fs = S.DeviceTree(t, ncrit, quad).fused(theta, 0.01, iblock)
    a32, p32 = run_fused(torch, fs, n)
    assert fs.totals() == (hl.n_list, hl.interactions, hl.cell_interactions)
    check_fp32(a32, p32, a64, p64)
    # run to run: identical
    a2, _ = run_fused(torch, fs, n)
    np.testing.assert_array_equal(a2, a32)


def test_fused_theta_zero_and_absolute_mac(torch):
    pos, mass = ic.plummer(6000, 62)
    t = S.Tree(pos, mass, 8)
    # theta = 0: every group's list is every particle (the direct sum)
    hl = t.lists(0.0, 64, 0.02, True)
    fs = S.DeviceTree(t, 64, True).fused(0.0, 0.02, 2)
    a32, p32 = run_fused(torch, fs, 6000)
    assert fs.totals()[1] == 6000 * 6000
    check_fp32(a32, p32, *fp64_on_host_lists(hl, 64))
    # the absolute MAC (Eq. SW_MAC)
    hl = t.lists(0.0, 64, 0.02, True, mac="sw", delta=1e-3, m_limit=0.05)
    fs = S.DeviceTree(t, 64, True, mac="sw", delta=1e-3, m_limit=0.05).fused(0.0, 0.02, 2)
    a32, p32 = run_fused(torch, fs, 6000)
    assert fs.totals() == (hl.n_list, hl.interactions, hl.cell_interactions)
    check_fp32(a32, p32, *fp64_on_host_lists(hl, 64))


def test_fused_per_group_angles(torch):
    pos, mass = ic.hernquist(12000, 63)
    t = S.Tree(pos, mass, 8)
    dt = S.DeviceTree(t, 64, True)
    th = np.full(dt.n_groups, 0.6, np.float32)
    th[::4] = -1.0   # skipped: no output
    th[1::4] = 0.0
    th[2::4] = 0.9
    hl = t.lists(0.5, 64, 0.01, True, theta_per_group=th)
    a64, p64 = fp64_on_host_lists(hl, 64)
    a32, p32 = run_fused(torch, dt.fused(0.5, 0.01, 2, theta_per_group=th), 12000)
    # the particles of skipped groups (tree order -> caller order) get no output
    g = hl.groups
    skipped = np.zeros(12000, bool)
    for k in np.nonzero(th < 0)[0]:
        skipped[hl.perm[g["first"][k]:g["first"][k] + g["count"][k]]] = True
    assert skipped.any() and np.array_equal(np.isnan(a32[:, 0]), skipped)
    check_fp32(a32[~skipped], p32[~skipped], a64[~skipped], p64[~skipped])


def test_fused_on_device_tree_matches_device_step(torch):
    pos, mass = ic.plummer(1 << 15, 64)
    dt = S.DeviceTree.build(pos, mass, 8, 64, True, "cuda")
    dl = dt.walk(0.5, 1e-3)
    tune = L.default_tune(64)
    a64, p64 = (x.cpu().numpy() for x in S.force(S.DeviceStep(dl, dl.plan(tune)), precision=L.OTOO_FP64))
    fs = dt.fused(0.5, 1e-3, 2)
    a32, p32 = run_fused(torch, fs, 1 << 15)
    assert fs.totals() == (dl.n_list, dl.interactions, dl.cell_interactions)
    check_fp32(a32, p32, a64, p64)


def test_fused_rejects_what_it_cannot_do(torch):
    pos, mass = ic.plummer(5000, 65)
    t = S.Tree(pos, mass, 8)
    # groups of up to 64 particles with one target per lane (at most 32)
    fs = S.DeviceTree(t, 64, True).fused(0.5, 0.01, 1)
    acc = torch.zeros((5000, 3), dtype=torch.float64, device="cuda")
    pot = torch.zeros(5000, dtype=torch.float64, device="cuda")
    with pytest.raises(L.OtooError) as ei:
        fs(acc, pot)
    assert ei.value.code == L.OTOO_EDEVICE
    # the SPH walk has no force; iblock outside {1, 2, 4}
    h = ic.sph_radii(pos, mass, 32, "plummer")
    sph = S.DeviceTree(t, 64, False, mac="sph", h_sph=h).fused(0.0, 0.01, 2)
    with pytest.raises(L.OtooError) as ei:
        sph(acc, pot)
    assert ei.value.code == L.OTOO_EINVAL
    bad = S.DeviceTree(t, 64, True).fused(0.5, 0.01, 3)
    with pytest.raises(L.OtooError) as ei:
        bad(acc, pot)
    assert ei.value.code == L.OTOO_EINVAL


def test_fused_keeps_the_softened_quadrupole_at_large_eps(torch):
    # eps = 0.3: the quadrupole's B_2 eps^2 part is large; the fused kernel
    # stages it as the split kernels do
    pos, mass = ic.plummer(4096, 71)
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.5, 64, 0.3, True)
    a64, p64 = fp64_on_host_lists(hl, 64)
    fs = S.DeviceTree(t, 64, True).fused(0.5, 0.3, 2)
    a32, p32 = run_fused(torch, fs, 4096)
    assert fs.totals() == (hl.n_list, hl.interactions, hl.cell_interactions)
    check_fp32(a32, p32, a64, p64)
