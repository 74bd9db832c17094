"""SPH density stage on the device (needs a GPU): the SPH walk's lists
(Eq. SPH_RAD) on the host and on the device, and the density kernel against
the oracle's direct sum rho_i = sum_j m_j W(|x_i - x_j|, h_j) (Eq. SPH_SUM):
relative error <= 1e-5 (FP32 pair terms, FP64 sums)."""
import numpy as np
import pytest

import oracle
from paper_1206_1199_gb300 import _lib as L
from paper_1206_1199_gb300 import ic, system as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    L.load()
    return t


def tune_for(ncrit, iblock=2, split=16384):
    t = L.default_tune(ncrit)
    t.iblock, t.split = iblock, split
    return t


@pytest.mark.parametrize("model,n,ncrit,iblock,split", [("plummer", 20000, 64, 2, 16384),
                                                        ("hernquist", 20000, 32, 1, 16384),
                                                        ("plummer", 8000, 128, 4, 200)])
def test_density_on_host_lists_matches_oracle(torch, model, n, ncrit, iblock, split):
    pos, mass = ic.make(model, n, 61)
    h = ic.sph_radii(pos, mass, 48, model)
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.0, ncrit, 1.0, False, mac="sph", h_sph=h)
    assert np.all(hl.groups["n_cell"] == 0)
    tune = tune_for(ncrit, iblock, split)
    plan = hl.plan(tune)
    if split < 1000:
        assert plan.n_splits > 0
    dev = S.DeviceSystem.upload(hl, plan, "cuda")
    rho = S.sph_density(dev, h).cpu().numpy()
    ref = oracle.sph_density(pos, mass, h.astype(np.float64))
    np.testing.assert_allclose(rho, ref, rtol=1e-5)
    # the tree pairs are the oracle walk's
    r = oracle.Tree(pos, mass, 8, ncrit).sph_density(h.astype(np.float64))
    assert hl.interactions == r["pairs"]


def test_density_self_only(torch):
    # radii far below the spacing: each particle sees only itself
    pos, mass = ic.plummer(3000, 62)
    h = np.full(3000, 1e-7, np.float32)
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.0, 64, 1.0, False, mac="sph", h_sph=h)
    # the lists still hold the particles of the leaves that touch each
    # group's box (W = 0 for all of them but the particle itself)
    assert hl.interactions < 0.1 * 3000 * 3000
    dev = S.DeviceSystem.upload(hl, hl.plan(tune_for(64)), "cuda")
    rho = S.sph_density(dev, h).cpu().numpy()
    np.testing.assert_allclose(rho, mass * 8 / (np.pi * h.astype(np.float64) ** 3), rtol=1e-6)


def test_device_walk_sph_lists_match_host(torch):
    pos, mass = ic.hernquist(30000, 63)
    h = ic.sph_radii(pos, mass, 64, "hernquist")
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.0, 64, 1.0, False, mac="sph", h_sph=h)
    dt = S.DeviceTree(t, 64, False, mac="sph", h_sph=h)
    dl = dt.walk(0.0, 1.0)
    gh, gd = hl.groups, dl.groups
    for k in ("first", "count", "n_cell", "n_part", "list_off"):
        np.testing.assert_array_equal(gd[k], gh[k])
    lh, ld = hl.list, dl.list
    for g in range(0, len(gh), 7):
        o, npt = gh["list_off"][g], gh["n_part"][g]
        np.testing.assert_array_equal(np.sort(ld[o:o + npt]), lh[o:o + npt])
    np.testing.assert_array_equal(dt.walk(0.0, 1.0, exact=True).list, dl.list)


@pytest.mark.parametrize("model", ["plummer", "hernquist"])
def test_density_whole_device_pipeline(torch, model):
    n = 1 << 15
    pos, mass = ic.make(model, n, 64)
    h = ic.sph_radii(pos, mass, 64, model)
    dt = S.DeviceTree.build(pos, mass, 8, 64, False, "cuda", mac="sph", h_sph=h)
    dl = dt.walk(0.0, 1.0)
    tune = tune_for(64)
    step = S.DeviceStep(dl, dl.plan(tune))
    rho = S.sph_density(step, h).cpu().numpy()
    ref = oracle.sph_density(pos, mass, h.astype(np.float64))
    np.testing.assert_allclose(rho, ref, rtol=1e-5)
    # r_SPH in the device records against the host tree's
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.0, 64, 1.0, False, mac="sph", h_sph=h)
    assert abs(dl.interactions - hl.interactions) <= 1e-4 * hl.interactions


def test_device_brute_force_matches_oracle(torch):
    pos, mass = ic.hernquist(6000, 65)
    h = ic.sph_radii(pos, mass, 64, "hernquist")
    tgt = ic.subsample(6000, 300, 2)
    rho = S.sph_direct(pos, mass, h, tgt)
    ref = oracle.sph_density(pos, mass, h.astype(np.float64), targets=tgt)
    np.testing.assert_allclose(rho, ref, rtol=1e-12)
