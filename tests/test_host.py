"""Host half of the C ABI (no GPU): the library loads and exports every
declared symbol; the tree, groups, lists, batch packing and plan keep their
invariants; the host walk reaches the same accept/open decisions as the
independently written oracle."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_1206_1199_gb300 import _lib as L
from paper_1206_1199_gb300 import ic, system as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_1206_1199_gb300 import build
    build.build()
    return L.load()


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(otoo_\w+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert "otoo_force" in names and "otoo_build_tree" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_struct_sizes_match_header():
    assert ctypes.sizeof(L.Src) == 32 and ctypes.sizeof(L.Quad) == 32 and ctypes.sizeof(L.Group) == 64
    assert ctypes.sizeof(L.Item) == 32 and ctypes.sizeof(L.Split) == 16
    assert ctypes.sizeof(L.WCell) == 64 and ctypes.sizeof(L.WCell64) == 96


C_STRUCTS = {"Params": "otoo_params", "Tune": "otoo_tune", "Src": "otoo_src", "Quad": "otoo_quad",
             "Group": "otoo_group", "Item": "otoo_item", "Split": "otoo_split", "DevSystem": "otoo_dev_system",
             "ListsView": "otoo_lists_view", "PlanInfo": "otoo_plan_info", "TreeView": "otoo_tree_view",
             "WCell": "otoo_wcell", "WCell64": "otoo_wcell64", "DevWalk": "otoo_dev_walk", "DevTree": "otoo_devtree",
             "ThetaNet": "otoo_theta_net", "ThetaRule": "otoo_theta_rule"}


def test_ctypes_layouts_match_the_c_header(tmp_path):
    # every struct the binding mirrors: size and every field's offset as a C
    # compiler lays out include/otoo.h (a field the header lacks fails to build)
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "otoo.h"', "int main(void) {"]
    expect = []
    for py, c in C_STRUCTS.items():
        cls = getattr(L, py)
        lines.append('printf("%%zu\\n", sizeof(%s));' % c)
        expect.append(ctypes.sizeof(cls))
        for f in cls._fields_:
            lines.append('printf("%%zu\\n", offsetof(%s, %s));' % (c, f[0]))
            expect.append(getattr(cls, f[0]).offset)
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]
    assert got == expect


def tree_and_lists(pos, mass, theta=0.5, n_crit=64, eps=0.01, quad=True, leaf=8):
    t = S.Tree(pos, mass, leaf)
    return t, t.lists(theta, n_crit, eps, quad)


@pytest.mark.parametrize("model,n,leaf", [("plummer", 5000, 8), ("hernquist", 20000, 8), ("uniform", 3000, 1)])
def test_tree_invariants(model, n, leaf):
    pos, mass = ic.make(model, n, 21)
    t = S.Tree(pos, mass, leaf)
    e = t.export()
    nc = e["n_cell"]
    assert np.array_equal(np.sort(e["perm"]), np.arange(n))
    np.testing.assert_array_equal(e["pos"], pos[e["perm"]])
    b, en, lev, nch, c0 = e["begin"], e["end"], e["level"], e["nchild"], e["child0"]
    assert b[0] == 0 and en[0] == n and lev[0] == 0
    leaves = nch == 0
    # every particle in exactly one leaf
    cover = np.zeros(n, np.int64)
    for c in np.nonzero(leaves)[0]:
        cover[b[c]:en[c]] += 1
    assert np.all(cover == 1)
    assert np.all((en[leaves] - b[leaves] <= leaf) | (lev[leaves] == 21))
    side = e["root_side"] / 2.0 ** lev
    for c in range(nc):
        # particles inside the cell's cube (closed interval, one grid step slack)
        lo = e["root_lo"] + e["org"][c] * e["root_side"] / 2.0 ** 21
        p = e["pos"][b[c]:en[c]]
        h = e["root_side"] / 2.0 ** 21
        assert np.all(p >= lo - h) and np.all(p <= lo + side[c] + h)
        m = e["mass"][b[c]:en[c]].astype(np.float64)
        assert abs(e["cmass"][c] - m.sum()) <= 1e-12 * m.sum()
        np.testing.assert_allclose(e["com"][c], (m[:, None] * p).sum(0) / m.sum(), rtol=0, atol=1e-12 * side[c])
        if nch[c]:
            kids = np.arange(c0[c], c0[c] + nch[c])
            assert b[kids[0]] == b[c] and en[kids[-1]] == en[c]
            assert np.all(en[kids[:-1]] == b[kids[1:]])
            assert np.all(lev[kids] == lev[c] + 1)


def test_cell_spread_matches_oracle():
    # B_2 (Eq. B2) and b_max of every cell against the oracle's own sum over
    # the cell's particles
    pos, mass = ic.hernquist(6000, 33)
    t = S.Tree(pos, mass, 8)
    e = t.export()
    for c in range(0, e["n_cell"], 7):
        p = e["pos"][e["begin"][c]:e["end"][c]]
        m = e["mass"][e["begin"][c]:e["end"][c]].astype(np.float64)
        b2, bmax, _ = oracle.sw_radius(p, m, 1.0)
        assert e["b2"][c] == pytest.approx(b2, rel=1e-12, abs=1e-300)
        assert e["bmax"][c] == pytest.approx(bmax, rel=1e-12, abs=1e-300)


def test_hilbert_order_is_spatially_local():
    # consecutive particles in tree order are close (Hilbert keys): the mean
    # step is far below that of a random order
    pos, mass = ic.uniform_sphere(20000, 22)
    t = S.Tree(pos, mass, 8)
    e = t.export()
    step = np.linalg.norm(np.diff(e["pos"], axis=0), axis=1).mean()
    rnd = np.linalg.norm(np.diff(pos, axis=0), axis=1).mean()
    assert step < 0.1 * rnd


def test_groups_and_list_mass_completeness():
    pos, mass = ic.hernquist(30000, 23)
    t, lists = tree_and_lists(pos, mass, 0.6, 64, 1e-3)
    g = lists.groups
    assert g["count"].sum() == 30000 and g["count"].max() <= 64
    assert np.all(np.diff(g["first"]) > 0) and g["first"][0] == 0
    np.testing.assert_array_equal(g["first"][1:], g["first"][:-1] + g["count"][:-1])
    src = lists.src
    lst = lists.list
    total = mass.astype(np.float64).sum()
    n = lists.n_part
    for k in range(0, lists.n_groups, max(1, lists.n_groups // 300)):
        off, nc, npart = g["list_off"][k], g["n_cell"][k], g["n_part"][k]
        ent = lst[off:off + nc + npart]
        assert np.all(ent[:nc] >= n) and np.all(ent[nc:] < n)
        # a cell is accepted OR its particles appear -- never both, never neither
        ex = t.export()
        parts = set(ent[nc:].tolist())
        for c in ent[:nc] - n:
            assert not parts.intersection(range(ex["begin"][c], ex["end"][c]))
        m = ex["cmass"][ent[:nc] - n].sum() + src["m"][ent[nc:]].astype(np.float64).sum()
        assert abs(m - total) <= 1e-5 * total
        # the group's own particles are all in its list
        assert parts.issuperset(range(g["first"][k], g["first"][k] + g["count"][k]))


def test_theta_zero_lists_are_all_particles():
    pos, mass = ic.plummer(1500, 24)
    _, lists = tree_and_lists(pos, mass, 0.0, 64)
    g = lists.groups
    assert np.all(g["n_cell"] == 0) and np.all(g["n_part"] == 1500)
    assert lists.interactions == 1500 * 1500


@pytest.mark.parametrize("model,n,theta,ncrit,leaf", [("plummer", 4096, 0.5, 64, 8), ("plummer", 20000, 0.3, 128, 8),
                                                      ("hernquist", 20000, 0.75, 32, 8), ("uniform", 8000, 0.5, 16, 4),
                                                      ("king", 6000, 0.9, 64, 1)])
def test_walk_decisions_match_oracle(model, n, theta, ncrit, leaf):
    pos, mass = ic.make(model, n, 25)
    t, lists = tree_and_lists(pos, mass, theta, ncrit, 0.01, True, leaf)
    r = oracle.Tree(pos, mass, leaf, ncrit).eval(theta, 0.01, True, group_stride=10 ** 9)
    assert lists.n_groups == len(r["key"])
    g = lists.groups
    perm = lists.perm
    keys = np.array([perm[a:a + c].min() for a, c in zip(g["first"], g["count"])])
    mine = {k: (c, nc, npt) for k, c, nc, npt in zip(keys, g["count"], g["n_cell"], g["n_part"])}
    theirs = {k: (c, nc, npt) for k, c, nc, npt in zip(r["key"], r["count"], r["n_cell"], r["n_part"])}
    assert mine.keys() == theirs.keys()
    diff = [k for k in mine if mine[k] != theirs[k]]
    # an accept/open decision may flip only at an exact FP64 tie (none expected here)
    assert len(diff) == 0, diff[:5]
    assert lists.interactions == r["interactions"] * 0 + sum(c * (nc + npt) for c, nc, npt in mine.values())


@pytest.mark.parametrize("model,n,delta,m_limit,ncrit", [("plummer", 8000, 1e-2, 0.05, 64),
                                                        ("plummer", 8000, 1e-4, 0.0, 32),
                                                        ("hernquist", 20000, 1e-3, 0.02, 128),
                                                        ("uniform", 6000, 3e-3, 0.05, 16)])
def test_sw_walk_decisions_match_oracle(model, n, delta, m_limit, ncrit):
    pos, mass = ic.make(model, n, 27)
    t = S.Tree(pos, mass, 8)
    lists = t.lists(0.0, ncrit, 0.01, True, mac="sw", delta=delta, m_limit=m_limit)
    r = oracle.Tree(pos, mass, 8, ncrit).eval(0.0, 0.01, True, group_stride=10 ** 9, mac="sw", delta=delta,
                                              m_limit=m_limit)
    g = lists.groups
    perm = lists.perm
    keys = np.array([perm[a:a + c].min() for a, c in zip(g["first"], g["count"])])
    mine = {k: (c, nc, npt) for k, c, nc, npt in zip(keys, g["count"], g["n_cell"], g["n_part"])}
    theirs = {k: (c, nc, npt) for k, c, nc, npt in zip(r["key"], r["count"], r["n_cell"], r["n_part"])}
    assert mine == theirs
    assert np.all(g["theta"] == 0)
    # no accepted cell is heavier than the mass limit
    if m_limit > 0:
        e = t.export()
        lst = lists.list
        cells = lst[lst >= lists.n_part] - lists.n_part
        assert e["cmass"][cells].max() <= m_limit


@pytest.mark.parametrize("model,n,ncrit,n_ngb", [("plummer", 8000, 64, 32), ("hernquist", 12000, 32, 64)])
def test_sph_walk_matches_oracle(model, n, ncrit, n_ngb):
    pos, mass = ic.make(model, n, 37)
    h = ic.sph_radii(pos, mass, n_ngb, model)
    t = S.Tree(pos, mass, 8)
    lists = t.lists(0.0, ncrit, 1.0, False, mac="sph", h_sph=h)
    r = oracle.Tree(pos, mass, 8, ncrit).sph_density(h.astype(np.float64))
    g = lists.groups
    assert np.all(g["n_cell"] == 0)
    perm = lists.perm
    keys = np.array([perm[a:a + c].min() for a, c in zip(g["first"], g["count"])])
    assert dict(zip(keys, g["n_part"])) == dict(zip(r["key"], r["n_part"]))
    assert lists.interactions == r["pairs"]
    with pytest.raises(L.OtooError):
        bad = h.copy()
        bad[3] = 0.0
        t.lists(0.0, ncrit, 1.0, False, mac="sph", h_sph=bad)


def test_per_group_theta_override():
    pos, mass = ic.plummer(8000, 26)
    t, base = tree_and_lists(pos, mass, 0.5, 64)
    th = np.full(base.n_groups, 0.5, np.float32)
    th[::3] = 0.0
    l2 = t.lists(0.9, 64, 0.01, True, theta_per_group=th)
    g0, g2 = base.groups, l2.groups
    assert np.all(g2["n_cell"][::3] == 0) and np.all(g2["n_part"][::3] == 8000)
    keep = np.ones(base.n_groups, bool)
    keep[::3] = False
    np.testing.assert_array_equal(g2["n_cell"][keep], g0["n_cell"][keep])
    np.testing.assert_array_equal(g2["theta"][::3], 0.0)


def test_batch_packing_rebases_indices():
    systems = ic.batch_systems(n_sys=6, log2_min=8, log2_max=11)
    per = [tree_and_lists(p, m, 0.5, 64, e)[1] for p, m, e in systems]
    B = S.Lists.pack(per)
    assert B.n_part == sum(l.n_part for l in per) and B.n_src == sum(l.n_src for l in per)
    assert B.interactions == sum(l.interactions for l in per)
    off = B.sys_part_off
    cell_base = B.n_part + np.cumsum([0] + [l.n_src - l.n_part for l in per])
    gb = 0
    for k, l in enumerate(per):
        g = B.groups[gb:gb + l.n_groups]
        assert np.all(g["sys"] == k)
        np.testing.assert_array_equal(g["first"], l.groups["first"] + off[k])
        for j in range(0, l.n_groups, max(1, l.n_groups // 20)):
            a = l.list[l.groups["list_off"][j]: l.groups["list_off"][j] + l.groups["n_cell"][j] + l.groups["n_part"][j]]
            b = B.list[g["list_off"][j]: g["list_off"][j] + g["n_cell"][j] + g["n_part"][j]]
            exp = np.where(a < l.n_part, a + off[k], a - l.n_part + cell_base[k])
            np.testing.assert_array_equal(b, exp)
            np.testing.assert_array_equal(B.src[b], l.src[a])
        np.testing.assert_array_equal(B.perm[off[k]:off[k + 1]], l.perm + off[k])
        gb += l.n_groups


@pytest.mark.parametrize("split", [64, 300, 100000])
def test_plan_covers_every_list_once(split):
    # every (target, list entry) pair of every group is in exactly one item:
    # the items of a group tile its particles x list-entries rectangle
    pos, mass = ic.plummer(10000, 27)
    _, lists = tree_and_lists(pos, mass, 0.4, 64)
    for ib in (1, 2, 4):
        tune = L.default_tune(64)
        tune.split, tune.iblock = split, ib
        p = lists.plan(tune)
        it = p.items
        g = lists.groups
        L_ = g["n_cell"] + g["n_part"]
        assert np.all(it["j1"] - it["j0"] <= split) and np.all(it["ni"] <= 32 * ib) and np.all(it["ni"] >= 1)
        cover = {}
        for r in it:
            cover.setdefault(int(r["g"]), []).append((int(r["i0"]), int(r["ni"]), int(r["j0"]), int(r["j1"]),
                                                      int(r["slot"])))
        assert sorted(cover) == list(range(lists.n_groups))
        nsplit_chunks = 0
        for gi, segs in cover.items():
            i_ranges = sorted({(a, b) for a, b, _, _, _ in segs})
            j_ranges = sorted({(c, d) for _, _, c, d, _ in segs})
            assert len(segs) == len(i_ranges) * len(j_ranges)
            assert i_ranges[0][0] == 0 and sum(b for _, b in i_ranges) == g["count"][gi]
            assert all(a[0] + a[1] == b[0] for a, b in zip(i_ranges, i_ranges[1:]))
            assert j_ranges[0][0] == 0 and j_ranges[-1][1] == L_[gi]
            assert all(a[1] == b[0] for a, b in zip(j_ranges, j_ranges[1:]))
            slots = {s for *_, s in segs}
            if len(j_ranges) == 1:
                assert slots == {-1}
            else:
                assert min(slots) >= 0 and len(slots) == len(j_ranges)
                nsplit_chunks += len(j_ranges)
        ni = it["ni"].astype(np.int64)
        assert np.all(np.diff(ni * (it["j1"] - it["j0"])) <= 0)  # longest first
        sp = p.splits
        assert sp["n_chunks"].sum() == nsplit_chunks
        assert p.partial_doubles == sp["n_chunks"].sum() * 4 * p.n_crit_max


def _chunk_cut(n, ib):
    """Restatement of the plan's particle-chunk rule: the cut of n targets
    into items that minimises the summed modelled warp time (pair steps of
    36 per target, 4 per staged entry of a 4096-entry list, 600 per item, 40
    per round of the pairwise subset merge), ties to the smaller last chunk."""
    def cost(s):
        nsub = 32 // ((s + ib - 1) // ib)
        return (4096 + nsub - 1) // nsub * ib * 36 + 4 * 4096 + 600 + (nsub - 1).bit_length() * 40
    best, last = [0], [0]
    for m in range(1, n + 1):
        c = [(best[m - s] + cost(s), s) for s in range(1, min(m, 32 * ib) + 1)]
        b = min(c)
        best.append(b[0])
        last.append(b[1])
    out = []
    while n:
        out.append(last[n])
        n -= last[n]
    return out


@pytest.mark.parametrize("ib", [1, 2, 4])
def test_plan_particle_chunks_follow_the_cut(ib):
    # the items of a group have the sizes of the cost-minimising cut, first
    # chunk at i0 = 0; a group of 26 at ib = 2 is cut 10 + 16 (5 lanes x 6
    # subsets and 8 lanes x 4 subsets: 31 of 32 lanes busy against 26 lanes
    # for one item of 13 x 2)
    assert _chunk_cut(26, 2) == [10, 16] and _chunk_cut(64, 2) == [64] and _chunk_cut(128, 2) == [64, 64]
    pos, mass = ic.plummer(20000, 29)
    _, lists = tree_and_lists(pos, mass, 0.5, 128)
    tune = L.default_tune(128)
    tune.iblock, tune.split = ib, 100000
    plan = lists.plan(tune)  # the items view borrows the plan's memory
    it = plan.items
    g = lists.groups
    per = {}
    for r in it:
        per.setdefault(int(r["g"]), []).append((int(r["i0"]), int(r["ni"])))
    memo = {}
    for gi, segs in per.items():
        n = int(g["count"][gi])
        if n not in memo:
            memo[n] = _chunk_cut(n, ib)
        assert [ni for _, ni in sorted(segs)] == memo[n], (gi, n, sorted(segs))
    assert sum(int(r["ni"]) for r in it) == int(g["count"].sum())


def test_invalid_inputs_return_einval():
    pos, mass = ic.plummer(100, 28)
    for bad_pos, bad_mass in ((pos * np.nan, mass), (pos, mass * 0), (pos, -mass)):
        with pytest.raises(L.OtooError) as e:
            S.Tree(bad_pos, bad_mass)
        assert e.value.code == L.OTOO_EINVAL
    t = S.Tree(pos, mass)
    for theta, ncrit, eps in ((-0.1, 64, 0.1), (0.5, 0, 0.1), (0.5, 5000, 0.1), (0.5, 64, 0.0), (0.5, 64, np.inf)):
        with pytest.raises(L.OtooError) as e:
            t.lists(theta, ncrit, eps)
        assert e.value.code == L.OTOO_EINVAL
    with pytest.raises(L.OtooError):
        L.call("otoo_build_tree", None, None, 0, None, None)
    for delta in (-1.0, np.inf, np.nan):
        with pytest.raises(L.OtooError) as e:
            t.lists(0.0, 64, 0.1, mac="sw", delta=delta)
        assert e.value.code == L.OTOO_EINVAL
    p = S._params(0.5, 8, 64, True, 0.1)
    p.mac = 7
    h = __import__("ctypes").c_void_p()
    with pytest.raises(L.OtooError) as e:
        L.call("otoo_make_groups_and_lists", t._h, __import__("ctypes").byref(p), __import__("ctypes").byref(h))
    assert e.value.code == L.OTOO_EINVAL


def test_features_are_finite_and_consistent():
    pos, mass = ic.hernquist(20000, 29)
    t, lists = tree_and_lists(pos, mass, 0.5, 64, 5e-4)
    f = lists.features(t)
    assert f.shape == (lists.n_groups, 5) and np.all(np.isfinite(f))
    g = lists.groups
    np.testing.assert_allclose(f[:, 0], np.log2(g["n_cell"] + g["n_part"]), rtol=1e-6)
    assert np.all((f[:, 3] >= 0) & (f[:, 3] <= 1))
    # the truncation estimate grows with the opening angle (accepted cells are
    # larger relative to their distance)
    f9 = t.lists(0.9, 64, 5e-4, True).features(t)
    assert np.median(f9[:, 4]) > np.median(f[:, 4]) + 0.5
    # with theta = 0 no cell is accepted: fraction 0, min distance and
    # truncation at their sentinels
    _, l0 = tree_and_lists(pos[:2000], mass[:2000], 0.0, 64, 5e-4)
    f0 = l0.features(S.Tree(pos[:2000], mass[:2000]))
    assert np.all(f0[:, 3] == 0) and np.all(f0[:, 1] == np.float32(3.0)) and np.all(f0[:, 4] == np.float32(-12.0))


@pytest.mark.parametrize("model,n,theta,ncrit,eps", [("hernquist", 20000, 0.9, 64, 5e-4), ("plummer", 8000, 0.5, 32, 1e-2),
                                                      ("polytrope_pair", 16000, 1.2, 128, 1e-4)])
def test_features_match_oracle(model, n, theta, ncrit, eps):
    # the library's list statistics against the oracle's restatement on its
    # own tree and walk, group by group (matched by lowest particle index)
    pos, mass = ic.make(model, n, 30)
    t, lists = tree_and_lists(pos, mass, theta, ncrit, eps)
    f = lists.features(t)
    g, perm = lists.groups, lists.perm
    keys = np.array([perm[a:a + c].min() for a, c in zip(g["first"], g["count"])])
    okey, of = oracle.Tree(pos, mass, 8, ncrit).features(theta, eps)
    order = np.argsort(okey)
    pos_in = np.searchsorted(okey[order], keys)
    assert np.array_equal(okey[order][pos_in], keys)
    ref = of[order][pos_in]
    np.testing.assert_array_equal(f[:, 0], ref[:, 0].astype(np.float32))
    np.testing.assert_allclose(f[:, 1:3], ref[:, 1:3], rtol=0, atol=2e-6)
    np.testing.assert_allclose(f[:, 3], ref[:, 3], rtol=0, atol=1e-6)
    np.testing.assert_allclose(f[:, 4], ref[:, 4], rtol=0, atol=2e-6)
    assert np.mean(ref[:, 3] > 0) > 0.5


def device_arrays(t, use_quad, mac="theta", delta=0.0, m_limit=0.0):
    e = t.export()
    n, nc = e["n_part"], e["n_cell"]
    src = np.empty(n + nc, np.dtype(L.Src))
    quad = np.empty(nc, np.dtype(L.Quad))
    cell = np.empty(nc, np.dtype(L.WCell))
    cell64 = np.empty(nc, np.dtype(L.WCell64))
    p = S._params(0.0, 8, 64, use_quad, 1.0, None, mac, delta, m_limit)
    L.call("otoo_tree_device_arrays", t._h, int(use_quad), ctypes.byref(p), src.ctypes.data, quad.ctypes.data,
           cell.ctypes.data, cell64.ctypes.data)
    return e, src, quad, cell, cell64


def test_sw_walk_records_carry_the_radius():
    pos, mass = ic.plummer(5000, 34)
    t = S.Tree(pos, mass, 8)
    e, _, _, cell, cell64 = device_arrays(t, 1, "sw", 1e-3, 0.05)
    for c in range(0, e["n_cell"], 5):
        p = e["pos"][e["begin"][c]:e["end"][c]]
        m = e["mass"][e["begin"][c]:e["end"][c]].astype(np.float64)
        rb = oracle.sw_radius(p, m, 1e-3, 0.05, e["root_side"])[2]
        assert cell64["rb"][c] == pytest.approx(rb, rel=1e-12)
        assert cell["rb"][c] == np.float32(cell64["rb"][c])
    assert np.all(cell64["rb"][e["cmass"] > 0.05] == 2 * e["root_side"])
    _, _, _, c0, c64 = device_arrays(t, 1, "sw", 0.0, 0.0)
    assert np.all(np.isinf(c64["rb"])) and np.all(np.isinf(c0["rb"]))
    _, _, _, c0, c64 = device_arrays(t, 1)
    assert np.all(c64["rb"] == 0) and np.all(c0["rb"] == 0)


def find_groups(t, n_crit):
    G = ctypes.c_int64()
    L.call("otoo_find_groups", t._h, n_crit, None, None, 0, ctypes.byref(G))
    first = np.empty(G.value, np.int32)
    count = np.empty(G.value, np.int32)
    L.call("otoo_find_groups", t._h, n_crit, first.ctypes.data, count.ctypes.data, G.value, ctypes.byref(G))
    return first, count


@pytest.mark.parametrize("use_quad", [0, 1])
def test_device_arrays_match_lists_and_geometry(use_quad):
    pos, mass = ic.hernquist(12000, 31)
    t, lists = tree_and_lists(pos, mass, 0.6, 48, 0.01, bool(use_quad))
    e, src, quad, cell, cell64 = device_arrays(t, use_quad)
    # the force step's sources are the ones the host lists carry
    np.testing.assert_array_equal(src.view(np.uint8), lists.src.view(np.uint8))
    np.testing.assert_array_equal(quad.view(np.uint8), lists.quad.view(np.uint8))
    first, count = find_groups(t, 48)
    np.testing.assert_array_equal(first, lists.groups["first"])
    np.testing.assert_array_equal(count, lists.groups["count"])
    # FP64 geometry: cube_lo = lo + org * h, side = h * 2^(21 - level), centre = cube_lo + side / 2
    h = e["root_side"] / 2097152.0
    lo = e["root_lo"][None, :] + e["org"].astype(np.float64) * h
    side = h * (2.0 ** (21 - e["level"])).astype(np.float64)
    np.testing.assert_array_equal(cell64["lo"], lo)
    np.testing.assert_array_equal(cell64["side"], side)
    np.testing.assert_array_equal(cell64["gc"], lo + (side / 2)[:, None])
    np.testing.assert_array_equal(cell64["com"], e["com"])
    # FP32 walk records
    com = e["com"]
    np.testing.assert_array_equal(cell["com_hi"], com.astype(np.float32))
    np.testing.assert_array_equal(cell["com_lo"], (com - cell["com_hi"].astype(np.float64)).astype(np.float32))
    assert np.all(np.abs(cell["com_hi"].astype(np.float64) + cell["com_lo"] - com) <= 2.0 ** -46 * np.abs(com))
    np.testing.assert_array_equal(cell["e"], (com - lo).astype(np.float32))
    assert np.all(cell["e"] >= 0) and np.all(cell["e"] <= cell["side"][:, None])
    gc = lo + (side / 2)[:, None]
    dd = com - gc
    s2 = dd[:, 0] * dd[:, 0] + dd[:, 1] * dd[:, 1] + dd[:, 2] * dd[:, 2]
    np.testing.assert_array_equal(cell["s"], np.sqrt(s2).astype(np.float32))
    np.testing.assert_array_equal(cell["side"], side.astype(np.float32))
    np.testing.assert_array_equal(cell["nchild"], e["nchild"])
    np.testing.assert_array_equal(cell["child0"], np.where(e["nchild"] > 0, e["child0"], 0))
    np.testing.assert_array_equal(cell["begin"], e["begin"])
    np.testing.assert_array_equal(cell["end"], e["end"])


def exact_accept(blo, bhi, cell64, theta):
    """The host walk's FP64 acceptance test for one box against every cell
    (numpy, the same operations in the same order)."""
    if not theta > 0:
        return np.zeros(len(cell64), bool)
    lo, side, com, gc = cell64["lo"], cell64["side"], cell64["com"], cell64["gc"]
    chi = lo + side[:, None]
    overlap = np.all((lo <= bhi) & (blo <= chi), axis=1)
    d = np.maximum(np.maximum(blo - com, 0.0), com - bhi)
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    e = com - gc
    s2 = (e[:, 0] * e[:, 0] + e[:, 1] * e[:, 1]) + e[:, 2] * e[:, 2]
    return ~overlap & (np.sqrt(d2) > side / theta + np.sqrt(s2))


def filter_accept(blo, bhi, cell, theta):
    """FP32 filter of the device walk, restated in numpy float32: +1 accept,
    0 reject, -1 undecided (the device then runs the FP64 test)."""
    f = np.float32
    c = (blo + bhi) * 0.5
    c32 = c.astype(f)
    cl32 = (c - c32.astype(np.float64)).astype(f)
    bl = (blo - c).astype(f)
    bh = (bhi - c).astype(f)
    B = np.maximum(np.abs(bl), np.abs(bh)).sum(dtype=f)
    A0 = np.abs(c32).sum(dtype=f)
    invth = f(1.0 / theta)
    u = (cell["com_hi"] - c32) + (cell["com_lo"] - cl32)
    side = cell["side"]
    thr = side * invth + cell["s"]
    A = A0 + np.abs(cell["com_hi"]).sum(1, dtype=f)
    K = np.abs(u).sum(1, dtype=f) + B + thr + side + A * f(2.0 ** -24)
    dl = K * f(2.0 ** -18)
    lo = u - cell["e"]
    hi = lo + side[:, None]
    if theta < 0.57:
        # below 1/sqrt(3) the device leaves the overlap part out
        sep = np.ones(len(cell), bool)
        ovl = np.zeros(len(cell), bool)
    else:
        sep = np.any((lo > bh + dl[:, None]) | (bl > hi + dl[:, None]), axis=1)
        ovl = np.all((lo < bh - dl[:, None]) & (bl < hi - dl[:, None]), axis=1)
    d = np.maximum(f(0), np.maximum(bl - u, u - bh))
    d2 = (d * d).sum(1, dtype=f)
    thr2 = thr * thr
    m = K * K * f(2.0 ** -16)
    out = np.full(len(cell), -1, np.int8)
    out[sep & (d2 > thr2 + m)] = 1
    out[sep & (d2 < thr2 - m)] = 0
    out[ovl] = 0
    return out


def exact_accept_sw(blo, bhi, cell64):
    com = cell64["com"]
    d = np.maximum(np.maximum(blo - com, 0.0), com - bhi)
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    return np.sqrt(d2) > cell64["rb"]


def filter_accept_sw(blo, bhi, cell):
    """FP32 filter of the device walk's absolute MAC, restated in numpy."""
    f = np.float32
    c = (blo + bhi) * 0.5
    c32 = c.astype(f)
    cl32 = (c - c32.astype(np.float64)).astype(f)
    bl = (blo - c).astype(f)
    bh = (bhi - c).astype(f)
    B = np.maximum(np.abs(bl), np.abs(bh)).sum(dtype=f)
    A = np.abs(c32).sum(dtype=f) + np.abs(cell["com_hi"]).sum(1, dtype=f)
    u = (cell["com_hi"] - c32) + (cell["com_lo"] - cl32)
    rb = cell["rb"]
    K = np.abs(u).sum(1, dtype=f) + B + rb + A * f(2.0 ** -24)
    d = np.maximum(f(0), np.maximum(bl - u, u - bh))
    d2 = (d * d).sum(1, dtype=f)
    m = K * K * f(2.0 ** -16)
    out = np.full(len(cell), -1, np.int8)
    with np.errstate(invalid="ignore"):
        out[d2 > rb * rb + m] = 1
        out[d2 < rb * rb - m] = 0
    out[np.isinf(rb)] = 0
    return out


@pytest.mark.parametrize("model,delta,m_limit", [("plummer", 1e-2, 0.05), ("hernquist", 1e-4, 0.0),
                                                 ("plummer", 0.0, 0.0)])
def test_fp32_sw_filter_never_contradicts_fp64(model, delta, m_limit):
    pos, mass = ic.make(model, 6000, 35)
    t = S.Tree(pos, mass, 8)
    e, _, _, cell, cell64 = device_arrays(t, 1, "sw", delta, m_limit)
    first, count = find_groups(t, 32)
    undecided = total = 0
    for gi in range(0, len(first), 3):
        p = e["pos"][first[gi]:first[gi] + count[gi]]
        blo, bhi = p.min(0), p.max(0)
        ex = exact_accept_sw(blo, bhi, cell64)
        fl = filter_accept_sw(blo, bhi, cell)
        dec = fl >= 0
        np.testing.assert_array_equal(fl[dec] == 1, ex[dec])
        undecided += int((~dec).sum())
        total += len(fl)
    assert undecided <= 0.01 * total


@pytest.mark.parametrize("model,n,theta", [("plummer", 6000, 0.5), ("hernquist", 6000, 0.75),
                                           ("lattice", 4096, 0.5), ("lattice", 4096, 1.0),
                                           ("hernquist", 6000, 0.3), ("plummer", 6000, 0.5773)])
def test_fp32_filter_never_contradicts_fp64(model, n, theta):
    """Wherever the FP32 filter decides, the FP64 test decides the same; the
    undecided share stays small.  The lattice puts many cells exactly on the
    acceptance threshold."""
    if model == "lattice":
        k = round(n ** (1 / 3))
        g = (np.arange(k) + 0.5) / k
        pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3) * 2.0 + 10.0
        mass = np.full(len(pos), 1.0 / len(pos), np.float32)
    else:
        pos, mass = ic.make(model, n, 32)
    t = S.Tree(pos, mass, 8)
    e, _, _, cell, cell64 = device_arrays(t, 1)
    first, count = find_groups(t, 32)
    undecided = total = 0
    for gi in range(0, len(first), 3):
        p = e["pos"][first[gi]:first[gi] + count[gi]]
        blo, bhi = p.min(0), p.max(0)
        ex = exact_accept(blo, bhi, cell64, theta)
        fl = filter_accept(blo, bhi, cell, theta)
        dec = fl >= 0
        np.testing.assert_array_equal(fl[dec] == 1, ex[dec])
        undecided += int((~dec).sum())
        total += len(fl)
    assert undecided <= 0.01 * total


def test_set_walk_union_with_masks_equals_group_walks():
    """The set walk's method on the CPU: one walk over runs of 8 consecutive
    groups, each stack entry carrying the mask of the groups for which its
    cells are still open, each visited cell tested with each masked group's
    own FP64 test, gives every group exactly its own walk's entries (the host
    lists, compared as sets), with fewer visited cells than the per-group
    walks together."""
    pos, mass = ic.hernquist(6000, 36)
    theta = 0.5
    t = S.Tree(pos, mass, 8)
    lists = t.lists(theta, 32, 0.01, True)
    e, _, _, _, cell64 = device_arrays(t, 1)
    g = lists.groups
    G, n = len(g), e["n_part"]
    nchild, child0, begin, end = e["nchild"], e["child0"], e["begin"], e["end"]
    lst = lists.list
    visits_union = visits_single = 0
    for s0 in range(0, G, 8):
        gs = list(range(s0, min(s0 + 8, G)))
        acc = [exact_accept(e["pos"][g["first"][k]:g["first"][k] + g["count"][k]].min(0),
                            e["pos"][g["first"][k]:g["first"][k] + g["count"][k]].max(0), cell64, theta) for k in gs]
        cells = [set() for _ in gs]
        parts = [set() for _ in gs]
        stack = [(0, (1 << len(gs)) - 1)]
        while stack:
            c, m = stack.pop()
            visits_union += 1
            visits_single += bin(m).count("1")
            rej = 0
            for j in range(len(gs)):
                if not (m >> j) & 1:
                    continue
                if acc[j][c]:
                    cells[j].add(n + c)
                elif nchild[c] == 0:
                    parts[j].update(range(begin[c], end[c]))
                else:
                    rej |= 1 << j
            if rej:
                for k in range(child0[c] + nchild[c] - 1, child0[c] - 1, -1):
                    stack.append((k, rej))
        for j, k in enumerate(gs):
            o, nc, npt = g["list_off"][k], g["n_cell"][k], g["n_part"][k]
            assert cells[j] == set(lst[o:o + nc].tolist()), k
            assert parts[j] == set(lst[o + nc:o + nc + npt].tolist()), k
    assert visits_union * 2 < visits_single
