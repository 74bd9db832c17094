"""The device walk and the device plan (needs a GPU).

The device walk must give every group the same cell entries and the same
particle entries as the host walk (bit-exact as sets: each acceptance
decision is the host's FP64 decision), the same group records and list
offsets; with every test forced to FP64 it must give the same lists in the
same order as with the FP32 filter.  The device plan must give the host
plan's items (as a multiset) and its split records exactly.  Forces on the
device lists: the FP64 form against the FP64 oracle tree (<= 1e-6, as for
the host lists) and the FP32 form against the FP32 form on the host lists
(summation order only)."""
import ctypes

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


GROUP_KEYS = ("first", "count", "n_cell", "n_part", "list_off", "eps2", "cx", "cy", "cz", "theta", "sys")


def compare_lists(hl, dl):
    gh, gd = hl.groups, dl.groups
    for k in GROUP_KEYS:
        np.testing.assert_array_equal(gd[k], gh[k], err_msg=k)
    assert dl.n_list == hl.n_list
    assert dl.interactions == hl.interactions and dl.cell_interactions == hl.cell_interactions
    lh, ld = hl.list, dl.list
    for g in range(len(gh)):
        o, nc, npt = gh["list_off"][g], gh["n_cell"][g], gh["n_part"][g]
        np.testing.assert_array_equal(np.sort(ld[o:o + nc]), np.sort(lh[o:o + nc]))
        np.testing.assert_array_equal(np.sort(ld[o + nc:o + nc + npt]), lh[o + nc:o + nc + npt])


def lattice(k, scale=2.0, shift=10.0):
    g = (np.arange(k) + 0.5) / k
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * scale + shift
    return pos, np.full(len(pos), 1.0 / len(pos), np.float32)


@pytest.mark.parametrize("model,n,theta,ncrit,leaf,quad", [
    ("plummer", 20000, 0.5, 64, 8, True), ("plummer", 20000, 0.3, 128, 8, True),
    ("hernquist", 30000, 0.75, 32, 8, True), ("king", 8000, 1.0, 64, 1, False),
    ("uniform", 10000, 0.5, 16, 4, True), ("lattice", 4096, 0.5, 64, 8, True)])
@pytest.mark.parametrize("group_set", [0, 1, 3, 8])
def test_device_walk_matches_host_lists(torch, model, n, theta, ncrit, leaf, quad, group_set):
    # group_set: consecutive groups one warp walks together (0: chosen by the library)
    pos, mass = lattice(16) if model == "lattice" else ic.make(model, n, 41)
    t = S.Tree(pos, mass, leaf)
    hl = t.lists(theta, ncrit, 0.01, quad)
    dt = S.DeviceTree(t, ncrit, quad)
    dl = dt.walk(theta, 0.01, group_set=group_set)
    compare_lists(hl, dl)
    # every test in FP64: the same lists in the same order
    de = dt.walk(theta, 0.01, exact=True, group_set=group_set)
    np.testing.assert_array_equal(de.list, dl.list)
    np.testing.assert_array_equal(de.groups.view(np.uint8), dl.groups.view(np.uint8))
    # run to run: identical
    np.testing.assert_array_equal(dt.walk(theta, 0.01, group_set=group_set).list, dl.list)


@pytest.mark.parametrize("model,n,delta,m_limit,ncrit", [("plummer", 20000, 1e-2, 0.05, 64),
                                                        ("hernquist", 30000, 1e-4, 0.0, 32),
                                                        ("plummer", 3000, 0.0, 0.0, 64)])
@pytest.mark.parametrize("group_set", [1, 8])
def test_device_walk_sw_matches_host_lists(torch, model, n, delta, m_limit, ncrit, group_set):
    pos, mass = ic.make(model, n, 46)
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.0, ncrit, 0.01, True, mac="sw", delta=delta, m_limit=m_limit)
    dt = S.DeviceTree(t, ncrit, True, mac="sw", delta=delta, m_limit=m_limit)
    dl = dt.walk(0.0, 0.01, group_set=group_set)
    compare_lists(hl, dl)
    de = dt.walk(0.0, 0.01, exact=True, group_set=group_set)
    np.testing.assert_array_equal(de.list, dl.list)
    if delta == 0.0:
        assert dl.interactions == n * n


def test_set_walk_equals_group_walk(torch):
    # the set walk against the per-group walk on a larger tree: identical
    # group records, entries equal as sets per group; one angle for all
    # groups, one angle per group (each group's own threshold), the absolute
    # MAC
    pos, mass = ic.hernquist(1 << 17, 49)
    t = S.Tree(pos, mass, 8)
    dt = S.DeviceTree(t, 128, True)
    dsw = S.DeviceTree(t, 128, True, mac="sw", delta=1e-3, m_limit=0.05)
    tpg = np.random.default_rng(5).choice(np.float32([0.4, 0.55, 0.7, 0.85, 1.0]), dt.n_groups).astype(np.float32)
    cases = [(dt, 0.5, None, 8), (dt, 0.9, None, 5), (dt, 0.5, None, 0), (dt, 0.5, tpg, 8), (dsw, 0.0, None, 8)]
    for tree, theta, per_group, gs in cases:
        a = tree.walk(theta, 5e-4, theta_per_group=per_group, group_set=gs)
        b = tree.walk(theta, 5e-4, theta_per_group=per_group, group_set=1)
        np.testing.assert_array_equal(a.groups.view(np.uint8), b.groups.view(np.uint8))
        la, lb, g = a.list, b.list, a.groups
        for k in range(len(g)):
            o, nc, npt = g["list_off"][k], g["n_cell"][k], g["n_part"][k]
            np.testing.assert_array_equal(np.sort(la[o:o + nc]), np.sort(lb[o:o + nc]))
            np.testing.assert_array_equal(np.sort(la[o + nc:o + nc + npt]), np.sort(lb[o + nc:o + nc + npt]))


@pytest.mark.parametrize("delta", [1e-2, 1e-3])
def test_sw_lists_force_matches_oracle(torch, delta):
    pos, mass = ic.plummer(1 << 14, 47)
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.0, 64, 1e-3, True, mac="sw", delta=delta, m_limit=0.05)
    dev = S.DeviceSystem.upload(hl, hl.plan(L.default_tune(64)), "cuda")
    a64, p64 = (x.cpu().numpy() for x in S.force(dev, precision=L.OTOO_FP64))
    r = oracle.Tree(pos, mass, 8, 64).eval(0.0, 1e-3, use_quad=True, mac="sw", delta=delta, m_limit=0.05)
    rel = np.linalg.norm(a64 - r["acc"], axis=1) / np.linalg.norm(r["acc"], axis=1)
    assert rel.max() <= 1e-6
    assert (np.abs(p64 - r["pot"]) / np.abs(r["pot"])).max() <= 1e-6


@pytest.mark.parametrize("mac", ["theta", "sw", "sph"])
@pytest.mark.parametrize("group_set", [1, 8])
def test_one_pass_walk_equals_two_pass(torch, mac, group_set):
    pos, mass = ic.hernquist(30000, 48)
    h = ic.sph_radii(pos, mass, 48, "hernquist") if mac == "sph" else None
    t = S.Tree(pos, mass, 8)
    dt = S.DeviceTree(t, 64, mac != "sph", mac=mac, delta=1e-3, m_limit=0.05, h_sph=h)
    two = dt.walk(0.6 if mac == "theta" else 0.0, 0.01, group_set=group_set)
    pool = S.BufferPool("cuda")
    first = dt.walk(0.6 if mac == "theta" else 0.0, 0.01, pool=pool, group_set=group_set)
    assert not first.one_pass
    ref_list, ref_groups = two.list, two.groups
    one = dt.walk(0.6 if mac == "theta" else 0.0, 0.01, pool=pool, group_set=group_set)
    assert one.one_pass and one.in_place
    # in place: each group's entries contiguous in its slot, cells reversed
    ccap, pcap = one.slots
    g = one.groups
    G = len(g)
    assert one.list_len == G * (ccap + pcap)
    np.testing.assert_array_equal(g["list_off"], np.arange(G) * (ccap + pcap) + ccap - g["n_cell"])
    for f in ("first", "count", "n_cell", "n_part", "eps2", "cx", "cy", "cz", "theta", "sys"):
        np.testing.assert_array_equal(g[f], ref_groups[f], err_msg=f)
    np.testing.assert_array_equal(one.list, ref_list)
    # the dense copy (otoo_walk_compact) is the two-pass walk's, byte for byte
    one.compact()
    assert not one.in_place and one.list_len == one.n_list
    np.testing.assert_array_equal(one.bufs["list"][:one.n_list].cpu().numpy(), ref_list)
    np.testing.assert_array_equal(one.groups.view(np.uint8), ref_groups.view(np.uint8))
    # slots too small: the walk notices and fills the list in a second pass
    key = (dt.n_groups, dt.mac)
    pool.meta[key] = (4, 4)
    small = dt.walk(0.6 if mac == "theta" else 0.0, 0.01, pool=pool, group_set=group_set)
    assert not small.one_pass and not small.in_place
    np.testing.assert_array_equal(small.list, ref_list)
    np.testing.assert_array_equal(small.groups.view(np.uint8), ref_groups.view(np.uint8))


def test_forces_on_in_place_lists(torch):
    # the one-pass walk's slots as the list of a force step: the FP64 form
    # equals the dense lists' (cell order differs: rounding only), the FP32
    # form within its bound, and a too-small slot pool falls back cleanly
    pos, mass = ic.hernquist(1 << 15, 49)
    t = S.Tree(pos, mass, 8)
    dt = S.DeviceTree(t, 64, True)
    tune = L.default_tune(64)
    tune.split, tune.packed, tune.tile = 700, 1, 128
    dense = dt.walk(0.5, 1e-3)
    d_step = S.DeviceStep(dense, dense.plan(tune))
    pool = S.BufferPool("cuda")
    dt.walk(0.5, 1e-3, pool=pool)
    one = dt.walk(0.5, 1e-3, pool=pool)
    assert one.in_place
    step = S.DeviceStep(one, one.plan(tune))
    assert step.struct.n_list == one.list_len > one.n_list
    rel = lambda a, b: np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    a64, p64 = (x.cpu().numpy() for x in S.force(step, precision=L.OTOO_FP64))
    r64, q64 = (x.cpu().numpy() for x in S.force(d_step, precision=L.OTOO_FP64))
    assert rel(a64, r64).max() <= 1e-12 and (np.abs(p64 - q64) / np.abs(q64)).max() <= 1e-12
    a32, p32 = (x.cpu().numpy() for x in S.force(step, precision=L.OTOO_FP32K, tune=tune))
    d = rel(a32, r64)
    assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4
    assert (np.abs(p32 - q64) / np.abs(q64)).max() <= 1e-5


@pytest.mark.parametrize("group_set", [0, 3, 8])
def test_device_walk_theta_zero_and_per_group(torch, group_set):
    # with several groups per warp, sets mix skipped groups, angle 0 and
    # different angles
    pos, mass = ic.plummer(3000, 42)
    t = S.Tree(pos, mass, 8)
    dt = S.DeviceTree(t, 64, True)
    d0 = dt.walk(0.0, 0.02, group_set=group_set)
    g = d0.groups
    assert np.all(g["n_cell"] == 0) and np.all(g["n_part"] == 3000) and d0.interactions == 3000 * 3000
    compare_lists(t.lists(0.0, 64, 0.02, True), d0)
    th = np.full(dt.n_groups, 0.6, np.float32)
    th[::4] = -1.0   # skipped groups: empty lists
    th[1::4] = 0.0
    th[2::4] = 0.9
    hl = t.lists(0.5, 64, 0.02, True, theta_per_group=th)
    dl = dt.walk(0.5, 0.02, theta_per_group=th, group_set=group_set)
    compare_lists(hl, dl)
    assert np.all(dl.groups["n_cell"][::4] == 0) and np.all(dl.groups["n_part"][::4] == 0)


@pytest.mark.parametrize("group_set", [0, 8])
def test_device_walk_edge_cases(torch, group_set):
    # one particle: its list is itself
    t = S.Tree(np.array([[0.3, -0.2, 0.1]]), np.array([1.0], np.float32), 8)
    dl = S.DeviceTree(t, 64, True).walk(0.5, 0.1, group_set=group_set)
    compare_lists(t.lists(0.5, 64, 0.1, True), dl)
    assert dl.n_list == 1
    # coincident particles: a last-level leaf larger than n_crit is cut into chunks
    pos = np.zeros((300, 3))
    pos[150:] = 1e-9
    pos[:10] += np.linspace(0, 1, 10)[:, None]
    mass = np.full(300, 1 / 300, np.float32)
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.5, 32, 0.01, True)
    assert hl.groups["count"].max() == 32
    compare_lists(hl, S.DeviceTree(t, 32, True).walk(0.5, 0.01, group_set=group_set))


@pytest.mark.parametrize("split,iblock", [(16384, 2), (300, 2), (129, 1), (700, 4)])
def test_device_plan_matches_host_plan(torch, split, iblock):
    pos, mass = ic.hernquist(20000, 43)
    t = S.Tree(pos, mass, 8)
    hl = t.lists(0.5, 128, 0.01, True)
    tune = L.default_tune(128)
    tune.split, tune.iblock = split, iblock
    hp = hl.plan(tune)
    dp = S.DeviceTree(t, 128, True).walk(0.5, 0.01).plan(tune)
    assert (dp.n_items, dp.n_splits, dp.n_crit_max, dp.partial_doubles) == \
        (hp.n_items, hp.n_splits, hp.n_crit_max, hp.partial_doubles)
    key = lambda it: np.sort(it.view(np.uint8).reshape(-1, 32).view(np.int64).view(
        [("a", np.int64), ("b", np.int64), ("c", np.int64), ("d", np.int64)]).reshape(-1))
    np.testing.assert_array_equal(key(dp.items), key(hp.items))
    np.testing.assert_array_equal(dp.splits.view(np.uint8), hp.splits.view(np.uint8))
    # launch order: the groups' cost classes (quarter octaves of the largest
    # item's ni * (j1 - j0)) never increase
    it = dp.items
    cost = it["ni"].astype(np.int64) * (it["j1"] - it["j0"])
    c0 = np.zeros(hl.n_groups, np.int64)
    np.maximum.at(c0, it["g"], cost)
    msb = np.floor(np.log2(c0[it["g"]])).astype(np.int64)
    frac = np.where(msb >= 2, c0[it["g"]] >> np.maximum(msb - 2, 0), c0[it["g"]] << np.maximum(2 - msb, 0)) & 3
    cls = np.minimum(4 * msb + frac, 127)
    assert np.all(np.diff(cls) <= 0)


@pytest.mark.parametrize("split", [16384, 400])
def test_device_step_forces(torch, split):
    n = 1 << 15
    pos, mass = ic.plummer(n, 44)
    t = S.Tree(pos, mass, 8)
    tune = L.default_tune(64)
    tune.split = split
    tune.packed, tune.tile = 1, 128
    hl = t.lists(0.5, 64, 1e-3, True)
    hdev = S.DeviceSystem.upload(hl, hl.plan(tune), "cuda")
    dl = S.DeviceTree(t, 64, True).walk(0.5, 1e-3)
    step = S.DeviceStep(dl, dl.plan(tune))
    r = oracle.Tree(pos, mass, 8, 64).eval(0.5, 1e-3, use_quad=True)
    a64, p64 = (x.cpu().numpy() for x in S.force(step, precision=L.OTOO_FP64))
    rel = lambda a, b: np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)
    assert rel(a64, r["acc"]).max() <= 1e-6
    assert (np.abs(p64 - r["pot"]) / np.abs(r["pot"])).max() <= 1e-6
    h64, _ = (x.cpu().numpy() for x in S.force(hdev, precision=L.OTOO_FP64))
    assert rel(a64, h64).max() <= 1e-12
    a32, p32 = (x.cpu().numpy() for x in S.force(step, precision=L.OTOO_FP32K))
    h32, hp32 = (x.cpu().numpy() for x in S.force(hdev, precision=L.OTOO_FP32K))
    d = rel(a32, h32)
    assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4
    assert (np.abs(p32 - hp32) / np.abs(hp32)).max() <= 1e-5
    a2, _ = (x.cpu().numpy() for x in S.force(step, precision=L.OTOO_FP32K))
    np.testing.assert_array_equal(a2, a32)


@pytest.mark.parametrize("group_set", [0, 8])
def test_walk_reports_bad_records_and_small_lists(torch, group_set):
    pos, mass = ic.plummer(5000, 45)
    t = S.Tree(pos, mass, 8)
    dt = S.DeviceTree(t, 64, True)
    dl = dt.walk(0.5, 0.01, group_set=group_set)
    w, b = dl.struct, dl.bufs
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # a list one entry too short: nothing written, status set
    L.call("otoo_walk_count", ctypes.byref(w), b["groups"].data_ptr(), st)
    short = torch.full((dl.n_list,), -7, dtype=torch.int32, device="cuda")
    L.call("otoo_walk_fill", ctypes.byref(w), b["groups"].data_ptr(), short.data_ptr(), dl.n_list - 1, st)
    with pytest.raises(L.OtooError) as ei:
        L.call("otoo_walk_check_status", ctypes.byref(w), st)
    assert ei.value.code == L.OTOO_EDEVICE
    assert bool((short == -7).all())
    # a child link out of range: the record is skipped and reported
    cell = dt.bufs["cell"].view(torch.int32).view(-1, 16)
    root_child0 = int(cell[0, 11])
    cell[0, 11] = dt.n_cell + 5
    with pytest.raises(L.OtooError) as ei:
        dt.walk(0.5, 0.01, group_set=group_set)
    assert ei.value.code == L.OTOO_EDEVICE
    cell[0, 11] = root_child0
    compare_lists(t.lists(0.5, 64, 0.01, True), dt.walk(0.5, 0.01, group_set=group_set))
