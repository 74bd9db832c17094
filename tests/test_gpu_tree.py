"""The tree built on the device against the host build (needs a GPU).

Bit-exact: the particle order (permutation, sources), the cells as
(level, first, last particle) with their children, the cubes (corner, side,
centre), the groups.  To rounding: the moments (the device combines children
bottom-up, the host sums each cell's particles).  End to end: lists walked on
the device tree equal the host walk's group by group (decisions can only
flip at FP64 ties of the slightly different centres of mass), and the FP64
forces match the oracle tree."""
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


def host_arrays(t, use_quad=True, mac="theta", delta=0.0, m_limit=0.0):
    e = t.export()
    nc = e["n_cell"]
    cell = np.empty(nc, np.dtype(L.WCell))
    cell64 = np.empty(nc, np.dtype(L.WCell64))
    p = S._params(0.0, t.leaf_size, 64, use_quad, 1.0, None, mac, delta, m_limit)
    L.call("otoo_tree_device_arrays", t._h, int(use_quad), ctypes.byref(p), None, None, cell.ctypes.data,
           cell64.ctypes.data)
    return e, cell, cell64


def dev_arrays(dt):
    b = dt.bufs
    return dict(src=b["src"].cpu().numpy().view(np.dtype(L.Src)), cell=b["cell"].cpu().numpy().view(np.dtype(L.WCell)),
                cell64=b["cell64"].cpu().numpy().view(np.dtype(L.WCell64)), level=b["level"].cpu().numpy(),
                perm=b["perm"].cpu().numpy(), first=b["first"].cpu().numpy(), count=b["count"].cpu().numpy(),
                quad=b["quad"].cpu().numpy().view(np.dtype(L.Quad)) if b["quad"] is not None else None)


def cell_map(e, d):
    """device cell index -> host cell index, through (level, first particle)."""
    host = {(int(lv), int(b)): k for k, (lv, b) in enumerate(zip(e["level"], e["begin"]))}
    return np.array([host[(int(lv), int(b))] for lv, b in zip(d["level"], d["cell"]["begin"])])


def check_tree(pos, mass, leaf, ncrit, use_quad=True, mac="theta", delta=0.0, m_limit=0.0):
    t = S.Tree(pos, mass, leaf)
    e, hcell, hcell64 = host_arrays(t, use_quad, mac, delta, m_limit)
    dt = S.DeviceTree.build(pos, mass, leaf, ncrit, use_quad, "cuda", mac, delta, m_limit)
    d = dev_arrays(dt)
    n = len(pos)
    assert dt.n_cell == e["n_cell"] and dt.depth == e["depth"]
    np.testing.assert_array_equal(dt.root_lo, e["root_lo"])
    assert dt.root_side == e["root_side"]
    # particle order and sources
    np.testing.assert_array_equal(d["perm"], e["perm"])
    np.testing.assert_array_equal(np.stack([d["src"]["x"][:n], d["src"]["y"][:n], d["src"]["z"][:n]], 1), e["pos"])
    np.testing.assert_array_equal(d["src"]["m"][:n], e["mass"])
    # cells: same ranges, levels, children (mapped), cubes
    m = cell_map(e, d)
    assert len(np.unique(m)) == len(m)
    dc, d64 = d["cell"], d["cell64"]
    np.testing.assert_array_equal(dc["end"], e["end"][m])
    np.testing.assert_array_equal(dc["nchild"], e["nchild"][m])
    for k in np.nonzero(dc["nchild"])[0]:
        kids = m[dc["child0"][k]:dc["child0"][k] + dc["nchild"][k]]
        np.testing.assert_array_equal(kids, np.arange(e["child0"][m[k]], e["child0"][m[k]] + e["nchild"][m[k]]))
    for f in ("lo", "side", "gc"):
        np.testing.assert_array_equal(d64[f], hcell64[f][m])
    # moments to rounding
    side = d64["side"]
    np.testing.assert_allclose(d["src"]["m"][n:], e["cmass"][m].astype(np.float32), rtol=1e-6)
    com = e["com"][m]
    assert np.all(np.abs(d64["com"] - com) <= 1e-13 * (side[:, None] + np.abs(com)))
    if use_quad:
        # FP32 copies of quadrupoles summed in another order: a few FP32
        # ulps of the cell's second-moment scale (3 B_2 bounds every entry),
        # and FP64 rounding of offsets from the centre of mass (m side^2)
        scale = np.abs(e["quad"][m]).max(1) + 3 * e["b2"][m] + 1e-6 * e["cmass"][m] * side ** 2
        qd = np.stack([d["quad"][k] for k in ("xx", "yy", "zz", "xy", "xz", "yz")], 1).astype(np.float64)
        assert np.all(np.abs(qd - e["quad"][m]) <= 1e-6 * scale[:, None])
    if mac == "sw":
        rb, rh = d64["rb"], hcell64["rb"][m]
        fin = np.isfinite(rb)
        np.testing.assert_array_equal(np.isfinite(rh), fin)
        # B_2 (Eq. B2) vanishes for a cell whose particles coincide (a single
        # particle); an FP64 sum leaves rounding noise of about M (2^-52 |x|)^2
        # there, which the fourth root of Eq. SW_MAC turns into r_b of about
        # (3 noise / delta)^(1/4).  Those cells agree to that bound, the
        # others to 1e-10.
        mag = np.abs(com).max(1) + side
        noise = e["cmass"][m] * (2.0 ** -50 * mag) ** 2
        tiny = e["b2"][m] <= noise
        np.testing.assert_allclose(rb[fin & ~tiny], rh[fin & ~tiny], rtol=1e-10)
        lim = (12 * noise / delta) ** 0.25 + 2.0 ** -48 * mag
        assert np.all(np.abs(rb - rh)[fin & tiny] <= lim[fin & tiny])
    # groups
    G = dt.n_groups
    hf = np.empty(G + 8, np.int32)
    hc = np.empty(G + 8, np.int32)
    ng = ctypes.c_int64()
    L.call("otoo_find_groups", t._h, ncrit, hf.ctypes.data, hc.ctypes.data, G + 8, ctypes.byref(ng))
    assert ng.value == G
    np.testing.assert_array_equal(d["first"], hf[:G])
    np.testing.assert_array_equal(d["count"], hc[:G])
    return t, dt, m


@pytest.mark.parametrize("model,n,leaf,ncrit", [("plummer", 20000, 8, 64), ("hernquist", 50000, 8, 128),
                                                ("uniform", 10000, 1, 16), ("king", 7000, 4, 32),
                                                ("plummer", 3000, 64, 16)])
def test_device_tree_matches_host(torch, model, n, leaf, ncrit):
    pos, mass = ic.make(model, n, 51)
    check_tree(pos, mass, leaf, ncrit)


@pytest.mark.parametrize("model,n,leaf", [("plummer", 20000, 8), ("hernquist", 30000, 8), ("plummer", 5000, 1)])
def test_device_tree_sph_radius_is_an_upper_bound(torch, model, n, leaf):
    # The device's SPH radius (Eq. SPH_RAD) is an FP32 bound: never below
    # the host's FP64 value, and above it by at most 2^-19 relative plus the
    # FP32 rounding of the centre of mass and the particles and the bounds
    # added for it (a few 2^-24 of the coordinates' magnitudes; the particles
    # lie within r_b of the centre)
    pos, mass = ic.make(model, n, 53)
    h = ic.sph_radii(pos, mass, 64, model).astype(np.float32)
    t = S.Tree(pos, mass, leaf)
    e = t.export()
    cell = np.empty(e["n_cell"], np.dtype(L.WCell))
    cell64 = np.empty(e["n_cell"], np.dtype(L.WCell64))
    p = S._params(0.0, leaf, 64, False, 1.0, None, "sph", h_sph=h)
    L.call("otoo_tree_device_arrays", t._h, 0, ctypes.byref(p), None, None, cell.ctypes.data, cell64.ctypes.data)
    dt = S.DeviceTree.build(pos, mass, leaf, 64, False, "cuda", mac="sph", h_sph=h)
    d = dev_arrays(dt)
    m = cell_map(e, d)
    rd, rh = d["cell64"]["rb"], cell64["rb"][m]
    com1 = np.abs(d["cell64"]["com"]).sum(1)
    assert np.all(rd >= rh)
    assert np.all(rd <= rh * (1 + 2.0 ** -19) + 2.0 ** -20 * (com1 + rh))
    np.testing.assert_array_equal(d["cell"]["rb"], rd.astype(np.float32))


def test_device_tree_edge_cases(torch):
    # one particle; coincident particles (a last-level leaf bigger than
    # n_crit and leaf_size); a tiny cell capacity that has to grow
    check_tree(np.array([[0.3, -0.2, 0.1]]), np.array([1.0], np.float32), 8, 64)
    pos = np.zeros((300, 3))
    pos[150:] = 1e-9
    pos[:10] += np.linspace(0, 1, 10)[:, None]
    check_tree(pos, np.full(300, 1 / 300, np.float32), 8, 32)
    pos, mass = ic.plummer(5000, 52)
    t = S.Tree(pos, mass, 8)
    dt = S.DeviceTree.build(pos, mass, 8, 64, cap_cell=16)
    assert dt.n_cell == t.export()["n_cell"]
    # invalid input is rejected
    bad = pos.copy()
    bad[7, 1] = np.nan
    with pytest.raises(L.OtooError) as ei:
        S.DeviceTree.build(bad, mass, 8, 64)
    assert ei.value.code == L.OTOO_EINVAL
    with pytest.raises(L.OtooError) as ei:
        S.DeviceTree.build(pos, np.zeros_like(mass), 8, 64)
    assert ei.value.code == L.OTOO_EINVAL


@pytest.mark.parametrize("delta,m_limit", [(1e-3, 0.05), (1e-5, 0.0)])
def test_device_tree_sw_records(torch, delta, m_limit):
    pos, mass = ic.hernquist(30000, 53)
    check_tree(pos, mass, 8, 64, mac="sw", delta=delta, m_limit=m_limit)


@pytest.mark.parametrize("mac,theta,delta", [("theta", 0.5, 0.0), ("theta", 0.75, 0.0), ("sw", 0.0, 1e-3)])
def test_device_tree_walk_and_force(torch, mac, theta, delta):
    n = 1 << 15
    pos, mass = ic.plummer(n, 54)
    eps = 1e-3
    t = S.Tree(pos, mass, 8)
    hl = t.lists(theta, 64, eps, True, mac=mac, delta=delta, m_limit=0.05)
    dt = S.DeviceTree.build(pos, mass, 8, 64, True, "cuda", mac, delta, 0.05)
    dl = dt.walk(theta, eps)
    gh, gd = hl.groups, dl.groups
    np.testing.assert_array_equal(gd["first"], gh["first"])
    same = (gd["n_cell"] == gh["n_cell"]) & (gd["n_part"] == gh["n_part"])
    assert same.mean() >= 0.999
    tune = L.default_tune(64)
    step = S.DeviceStep(dl, dl.plan(tune))
    a64, p64 = (x.cpu().numpy() for x in S.force(step, precision=L.OTOO_FP64))
    r = oracle.Tree(pos, mass, 8, 64).eval(theta, eps, use_quad=True, mac=mac, delta=delta, m_limit=0.05)
    rel = np.linalg.norm(a64 - r["acc"], axis=1) / np.linalg.norm(r["acc"], axis=1)
    assert rel.max() <= 1e-6
    a32, _ = (x.cpu().numpy() for x in S.force(step, precision=L.OTOO_FP32K))
    sub = ic.subsample(n, 2048, 3)
    ad, _ = oracle.direct(pos, mass, eps, targets=sub)
    e = oracle.errors(a32[sub], np.zeros(len(sub)), ad, np.ones(len(sub)))
    assert e["acc_rms"] <= 2e-3
