"""Parity of the CUDA force path with the FP64 CPU oracle (needs a GPU).

Tolerances: the FP64 device form reproduces the oracle's tree force up to
summation order (<= 1e-6 max relative, expected ~1e-13); the FP32 form has
the tree error of theta plus FP32 rounding (<= 2e-3 RMS against the direct
sum at theta = 0.5) and differs from the FP64 form by FP32 rounding only
(<= 1e-5 max relative on accelerations)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1206_1199_gb300 import _lib as L
from paper_1206_1199_gb300 import autotune, ic, system as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    L.load()
    return t


def run(pos, mass, theta, n_crit, eps, use_quad, precision, tune=None, leaf=8):
    tree, lists, plan = S.build_system(pos, mass, theta, n_crit, eps, leaf, use_quad, tune)
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    a, p = S.force(dev, precision=precision)
    return a.cpu().numpy(), p.cpu().numpy(), lists


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def abs_sum(pos, mass, eps, centre):
    """Per target: sum over sources of |a_ij| and |phi_ij| (j != i), and the
    sensitivities of a_ij and phi_ij to the rounding of centre-relative FP32
    coordinates: m_j (D_i + D_j) / (r^2 + eps^2)^(3/2) and m_j (D_i + D_j) /
    (r^2 + eps^2), with D the distance to the group centre.  A sum's rounding
    error is a few ulps of the first pair of sums (not of |sum|, which is far
    smaller where the pulls cancel); coordinate rounding adds a few ulps of
    the second pair."""
    d = pos[None, :, :] - pos[:, None, :]
    d2 = (d * d).sum(-1)
    r2 = d2 + eps * eps
    m = np.broadcast_to(mass.astype(np.float64)[None, :], r2.shape).copy()
    np.fill_diagonal(m, 0.0)
    D = np.linalg.norm(pos - centre, axis=1)
    DD = D[:, None] + D[None, :]
    return ((m * np.sqrt(d2) / r2 ** 1.5).sum(1), (m / np.sqrt(r2)).sum(1),
            (m * DD / r2 ** 1.5).sum(1), (m * DD / r2).sum(1))


def within_bound(a, p, ad, pd, pos, mass, eps, k, centre=None):
    """|a - a_ref| <= k * sum_j |a_ij| + 8 u * coordinate sensitivity (u = 2^-24
    for the FP32 form, 0 for FP64) and the same for phi, per target."""
    c = (pos.min(0) + pos.max(0)) / 2 if centre is None else centre
    sa, sp, ca, cp = abs_sum(pos, mass, eps, c)
    u = 8 * 2.0 ** -24 if k > 1e-10 else 0.0
    return bool((np.linalg.norm(a - ad, axis=1) <= k * sa + u * ca).all() and (np.abs(p - pd) <= k * sp + u * cp).all())


# FP32 pair arithmetic: sums carry ~2^-24 rounding per term; accumulated over
# a list with Kahan sums the error stays a few 1e-7 of sum_j |a_ij|.
FP32_K = 2e-6


@pytest.mark.parametrize("quad", [False, True])
def test_fp64_matches_oracle_tree_plummer4k(torch, quad):
    pos, mass = ic.plummer(4096, ic.BASE_SEED + 1)
    a, p, _ = run(pos, mass, 0.5, 64, 0.01, quad, L.OTOO_FP64)
    r = oracle.Tree(pos, mass, 8, 64).eval(0.5, 0.01, use_quad=quad)
    assert rel(a, r["acc"]).max() <= 1e-6
    assert (np.abs(p - r["pot"]) / np.abs(r["pot"])).max() <= 1e-6
    # plus: the tree error of this configuration against the direct sum
    ad, pd = oracle.direct(pos, mass, 0.01)
    e = oracle.errors(a, p, ad, pd)
    assert e["acc_rms"] < (1e-3 if quad else 3e-3)


@pytest.mark.parametrize("theta", [0.3, 0.5, 0.75])
def test_fp32k_and_fp64_vs_oracle_plummer(torch, theta):
    n = 1 << 16
    pos, mass = ic.plummer(n, ic.BASE_SEED + 2)
    a64, p64, lists = run(pos, mass, theta, 128, 1e-3, True, L.OTOO_FP64)
    a32, p32, _ = run(pos, mass, theta, 128, 1e-3, True, L.OTOO_FP32K)
    r = oracle.Tree(pos, mass, 8, 128).eval(theta, 1e-3, use_quad=True)
    assert rel(a64, r["acc"]).max() <= 1e-6
    # FP32 vs FP64 on identical lists: arithmetic error only (RMS; the
    # largest per-particle value is set by cancelling pulls, see abs_sum)
    d = rel(a32, a64)
    assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4
    assert (np.abs(p32 - p64) / np.abs(p64)).max() <= 1e-5
    sub = ic.subsample(n, 4096, 7)
    ad, pd = oracle.direct(pos, mass, 1e-3, targets=sub)
    e = oracle.errors(a32[sub], p32[sub], ad, pd)
    if theta <= 0.5:
        assert e["acc_rms"] <= 2e-3


def test_tiny_direct_one_group(torch):
    # theta = 0, a single group: every pair is evaluated, both precisions
    pos, mass = ic.plummer(200, 3)
    ad, pd = oracle.direct(pos, mass, 0.05)
    for prec, k in ((L.OTOO_FP64, 1e-13), (L.OTOO_FP32K, FP32_K)):
        a, p, lists = run(pos, mass, 0.0, 256, 0.05, True, prec)
        assert lists.n_groups == 1
        assert within_bound(a, p, ad, pd, pos, mass, 0.05, k)


def test_theta0_many_groups_ragged(torch):
    # theta = 0 with groups of every size: lists of all n entries, j-split and
    # chunked lists (split below the list length) must all give the direct sum
    pos, mass = ic.hernquist(3001, 4)
    ad, pd = oracle.direct(pos, mass, 0.02)
    for split in (100000, 700, 129):
        tune = L.default_tune(64)
        tune.split = split
        for prec, k in ((L.OTOO_FP64, 1e-13), (L.OTOO_FP32K, FP32_K)):
            a, p, lists = run(pos, mass, 0.0, 64, 0.02, False, prec, tune=tune)
            assert within_bound(a, p, ad, pd, pos, mass, 0.02, k), (split, prec)


@pytest.mark.parametrize("block,iblock,tile,packed", [(128, 1, 128, 0), (128, 2, 64, 0), (128, 2, 256, 0),
                                                      (128, 4, 128, 0), (64, 4, 128, 0), (256, 2, 128, 0),
                                                      (128, 2, 128, 1), (64, 2, 128, 1), (128, 1, 128, 1),
                                                      (128, 2, 256, 1)])
def test_tuning_invariance(torch, block, iblock, tile, packed):
    pos, mass = ic.plummer(20000, 5)
    ref, refp, _ = run(pos, mass, 0.6, 64, 1e-2, True, L.OTOO_FP64)
    tune = L.Tune(block=block, iblock=iblock, tile=tile, split=max(tile, 300), ctas_per_sm=0, packed=packed)
    for prec in (L.OTOO_FP64, L.OTOO_FP32K):
        a, p, _ = run(pos, mass, 0.6, 64, 1e-2, True, prec, tune=tune)
        a2, p2, _ = run(pos, mass, 0.6, 64, 1e-2, True, prec, tune=tune)
        np.testing.assert_array_equal(a, a2)  # run to run: bit-identical
        d = rel(a, ref)
        if prec == L.OTOO_FP64:
            assert d.max() <= 1e-10
        else:
            assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4


def test_edge_cases(torch):
    # one particle: its list is itself, the self pair is removed exactly
    a, p, lists = run(np.array([[0.3, -0.2, 0.1]]), np.array([1.0], np.float32), 0.5, 64, 0.1, True, L.OTOO_FP64)
    assert lists.n_groups == 1 and np.all(a == 0) and abs(p[0]) < 1e-14
    # coincident particles: softening keeps them finite
    pos = np.zeros((40, 3))
    pos[20:] = 1e-9
    mass = np.full(40, 0.025, np.float32)
    ad, pd = oracle.direct(pos, mass, 0.01)
    for prec in (L.OTOO_FP64, L.OTOO_FP32K):
        a, p, _ = run(pos, mass, 0.5, 16, 0.01, True, prec)
        assert np.all(np.isfinite(a)) and np.allclose(p, pd, rtol=1e-5)
    # invalid inputs are rejected on the host with OTOO_EINVAL
    with pytest.raises(L.OtooError) as ei:
        S.build_system(np.array([[0.0, 0, 0], [1, 0, 0]]), np.ones(2, np.float32), 0.5, 64, 0.0)
    assert ei.value.code == L.OTOO_EINVAL
    with pytest.raises(L.OtooError):
        S.build_system(np.array([[np.nan, 0, 0], [1, 0, 0]]), np.ones(2, np.float32), 0.5, 64, 0.1)


def test_corrupt_list_index_is_reported(torch):
    # an out-of-range list entry is caught by the kernel's bounds check (the
    # entry is skipped) and reported as OTOO_EDEVICE; nothing is read out of range
    pos, mass = ic.plummer(2000, 6)
    tree, lists, plan = S.build_system(pos, mass, 0.5, 64, 0.01)
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    bad = lists.list.copy()
    bad[5] = 1 << 30
    dev.bufs["list"].copy_(torch.from_numpy(bad.view(np.uint8)).cuda())
    with pytest.raises(L.OtooError) as ei:
        S.force(dev, precision=L.OTOO_FP32K)
    assert ei.value.code == L.OTOO_EDEVICE


def test_outputs_in_pinned_host_memory(torch):
    # accel and pot in pinned host memory: the kernels write them there
    # directly, with the same bits as into device memory
    pos, mass = ic.plummer(30000, 9)
    tree, lists, plan = S.build_system(pos, mass, 0.5, 64, 1e-2)
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    n = lists.n_part
    for prec in (L.OTOO_FP32K, L.OTOO_FP64):
        a, p = S.force(dev, precision=prec)
        ah = torch.full((n, 3), np.nan, dtype=torch.float64).pin_memory()
        ph = torch.full((n,), np.nan, dtype=torch.float64).pin_memory()
        S.force(dev, ah, ph, precision=prec)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ah.numpy(), a.cpu().numpy())
        np.testing.assert_array_equal(ph.numpy(), p.cpu().numpy())


def test_host_entry_point_matches_device(torch):
    pos, mass = ic.plummer(30000, 8)
    tree, lists, plan = S.build_system(pos, mass, 0.5, 64, 1e-2)
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    a, p = S.force(dev, precision=L.OTOO_FP32K)
    ah, ph = S.force_host(lists, plan, precision=L.OTOO_FP32K)
    np.testing.assert_array_equal(a.cpu().numpy(), ah)
    np.testing.assert_array_equal(p.cpu().numpy(), ph)
    # pinned outputs (written by the kernel in place): the same bits
    n = lists.n_part
    ap = torch.full((n, 3), np.nan, dtype=torch.float64).pin_memory()
    pp = torch.full((n,), np.nan, dtype=torch.float64).pin_memory()
    S.force_host(lists, plan, precision=L.OTOO_FP32K, accel=ap, pot=pp)
    np.testing.assert_array_equal(ap.numpy(), ah)
    np.testing.assert_array_equal(pp.numpy(), ph)


def test_batch_packed_equals_separate(torch):
    systems = ic.batch_systems(n_sys=12, log2_min=8, log2_max=12)
    per = []
    for pos, mass, eps in systems:
        tree = S.Tree(pos, mass, 8)
        per.append((tree, tree.lists(0.5, 64, eps, True)))
    packed = S.Lists.pack([l for _, l in per])
    tune = L.default_tune(64)
    dev = S.DeviceSystem.upload(packed, packed.plan(tune), "cuda")
    for prec in (L.OTOO_FP64, L.OTOO_FP32K):
        a, p = S.force(dev, precision=prec)
        a, p = a.cpu().numpy(), p.cpu().numpy()
        off = packed.sys_part_off
        for k, (tree, lists) in enumerate(per):
            d = S.DeviceSystem.upload(lists, lists.plan(tune), "cuda")
            ak, pk = S.force(d, precision=prec)
            np.testing.assert_array_equal(a[off[k]:off[k + 1]], ak.cpu().numpy())
            np.testing.assert_array_equal(p[off[k]:off[k + 1]], pk.cpu().numpy())
    # per-system error against each system's own direct sum
    a, p = S.force(dev, precision=L.OTOO_FP32K)
    a = a.cpu().numpy()
    for k, (pos, mass, eps) in enumerate(systems):
        ad, _ = oracle.direct(pos, mass, eps)
        assert np.sqrt(np.mean(rel(a[off[k]:off[k + 1]], ad) ** 2)) < 2e-3


def test_partial_slots_past_the_buffer_are_reported(torch):
    # a work item or a split record whose partial slots reach past
    # sys.partial_doubles (a stale plan, a wrong size) is skipped and reported
    # as OTOO_EDEVICE; guard values after the buffer stay as they were
    pos, mass = ic.plummer(6000, 9)
    tune = L.default_tune(64)
    tune.split = 300
    tree, lists, plan = S.build_system(pos, mass, 0.5, 64, 1e-2, tune=tune)
    assert plan.n_splits > 0
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    need = plan.partial_doubles
    per_slot = 4 * plan.n_crit_max
    n_slots = need // per_slot
    assert n_slots * per_slot == need
    sentinel = 12345.0
    buf = torch.full((need + 8 * per_slot,), sentinel, dtype=torch.float64, device="cuda")
    dev.struct.partial = buf.data_ptr()
    dev.struct.partial_doubles = need
    ref, _ = S.force(dev, precision=L.OTOO_FP32K)  # the healthy plan passes its status check
    items = plan.items.copy()
    k = int(np.nonzero(items["slot"] >= 0)[0][0])
    items["slot"][k] = n_slots  # one slot past the end
    bad_items = torch.from_numpy(items.view(np.uint8).copy()).cuda()
    dev.struct.items = bad_items.data_ptr()
    for prec in (L.OTOO_FP32K, L.OTOO_FP64):
        with pytest.raises(L.OtooError) as ei:
            S.force(dev, precision=prec)
        assert ei.value.code == L.OTOO_EDEVICE
        assert bool(torch.all(buf[need:] == sentinel))
    dev.struct.items = dev.bufs["items"].data_ptr()
    splits = plan.splits.copy()
    splits["slot0"][0] = n_slots - splits["n_chunks"][0] + 1  # its last chunk lies past the end
    bad_splits = torch.from_numpy(splits.view(np.uint8).copy()).cuda()
    dev.struct.splits = bad_splits.data_ptr()
    with pytest.raises(L.OtooError) as ei:
        S.force(dev, precision=L.OTOO_FP32K)
    assert ei.value.code == L.OTOO_EDEVICE
    assert bool(torch.all(buf[need:] == sentinel))
    dev.struct.splits = dev.bufs["splits"].data_ptr()
    # too small a buffer for any split list is refused before launch
    dev.struct.partial_doubles = per_slot - 1
    with pytest.raises(L.OtooError) as ei:
        S.force(dev, precision=L.OTOO_FP32K)
    assert ei.value.code == L.OTOO_EINVAL
    dev.struct.partial_doubles = need
    a, _ = S.force(dev, precision=L.OTOO_FP32K)
    assert torch.equal(a, ref)


def test_autotuner_search_on_a_small_system(torch):
    # the coordinate descent itself: every visited variant times finite, the
    # returned tune is the fastest one it visited (each stage keeps the
    # current point among its candidates), and forces with it stay within
    # the FP32 bounds of the FP64 form
    pos, mass = ic.plummer(1 << 15, 10)
    w = dict(leaf_size=8, theta=0.5, eps=1e-2, use_quad=True)
    best, table = autotune.search(pos, mass, w, n_crits=(32, 64), log=lambda s: None)
    assert len(table) >= 10 and all(np.isfinite(r["ms"]) and r["ms"] > 0 for r in table)
    assert {r["n_crit"] for r in table} == {32, 64}
    assert best["ms"] == min(r["ms"] for r in table)
    assert (best["tune"]["block"], best["tune"]["iblock"], best["tune"]["tile"],
            best["tune"]["packed"]) in autotune.VARIANTS
    tune = L.Tune(**best["tune"])
    a32, _, lists = run(pos, mass, 0.5, best["n_crit"], 1e-2, True, L.OTOO_FP32K, tune=tune)
    a64, _, _ = run(pos, mass, 0.5, best["n_crit"], 1e-2, True, L.OTOO_FP64, tune=tune)
    d = rel(a32, a64)
    assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4


@pytest.mark.parametrize("packed", [0, 1])
def test_every_form_keeps_the_softened_quadrupole_at_large_eps(torch, packed):
    # eps = 0.3 on a Plummer sphere: the B_2 eps^2 part of the quadrupole term
    # moves the tree force by about 1e-3 (the batch configuration's regime),
    # so the FP64 form must match the oracle tree to 1e-6 and the scalar and
    # packed FP32 forms the FP64 form to their arithmetic bounds
    pos, mass = ic.plummer(4096, 71)
    eps = 0.3
    r = oracle.Tree(pos, mass, 8, 64).eval(0.5, eps, use_quad=True)
    a64, p64, lists = run(pos, mass, 0.5, 64, eps, True, L.OTOO_FP64)
    assert lists.cell_interactions > 0.3 * lists.interactions
    assert rel(a64, r["acc"]).max() <= 1e-6
    assert (np.abs(p64 - r["pot"]) / np.abs(r["pot"])).max() <= 1e-6
    tune = L.Tune(block=128, iblock=2, tile=128, split=100000, ctas_per_sm=0, packed=packed)
    a32, p32, _ = run(pos, mass, 0.5, 64, eps, True, L.OTOO_FP32K, tune=tune)
    d = rel(a32, a64)
    assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4
    assert (np.abs(p32 - p64) / np.abs(p64)).max() <= 1e-5


@pytest.mark.parametrize("iblock", [1, 2, 4])
def test_largest_groups(torch, iblock):
    # n_crit at its maximum (1024 particles per group): groups are cut into
    # work items of at most 32 iblock particles; every form against the
    # oracle tree (FP64) and the FP64 form (FP32, scalar and packed)
    pos, mass = ic.plummer(12000, 72)
    tree = S.Tree(pos, mass, 8)
    lists = tree.lists(0.5, 1024, 0.01, True)
    assert lists.groups["count"].max() > 512
    r = oracle.Tree(pos, mass, 8, 1024).eval(0.5, 0.01, use_quad=True)
    tune = L.Tune(block=128, iblock=iblock, tile=128, split=4096, ctas_per_sm=0, packed=0)
    dev = S.DeviceSystem.upload(lists, lists.plan(tune), "cuda")
    a64, p64 = (x.cpu().numpy() for x in S.force(dev, precision=L.OTOO_FP64, tune=tune))
    assert rel(a64, r["acc"]).max() <= 1e-6
    for packed in ((0, 1) if iblock < 4 else (0,)):
        t32 = L.Tune(block=128, iblock=iblock, tile=128, split=4096, ctas_per_sm=0, packed=packed)
        d32 = S.DeviceSystem.upload(lists, lists.plan(t32), "cuda")
        a32, _ = S.force(d32, precision=L.OTOO_FP32K, tune=t32)
        d = rel(a32.cpu().numpy(), a64)
        assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4, (iblock, packed)
