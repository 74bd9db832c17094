"""Pins of the FP64 oracle against closed forms, invariants and analytic
models (no GPU).  A plausible slip in the oracle -- a dropped term, a wrong
sign or index, a transposed operand -- breaks at least one of these."""
import math

import numpy as np
import pytest

import oracle
from golden_io import GOLDEN, load_bodies
from paper_1206_1199_gb300 import ic


@pytest.mark.parametrize("name", ["two_body.txt", "three_body.txt"])
def test_direct_closed_form(name):
    pos, mass, acc_ref, pot_ref, eps = load_bodies(name)
    acc, pot = oracle.direct(pos, mass, eps)
    np.testing.assert_allclose(acc, acc_ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(pot, pot_ref, rtol=1e-12, atol=0)


def test_direct_targets_subset_and_self_excluded():
    pos, mass = ic.plummer(300, 11)
    acc, pot = oracle.direct(pos, mass, 0.05)
    tgt = np.array([5, 17, 299])
    a2, p2 = oracle.direct(pos, mass, 0.05, targets=tgt)
    np.testing.assert_array_equal(a2, acc[tgt])
    np.testing.assert_array_equal(p2, pot[tgt])
    # the self pair would add exactly -m_i / eps to phi_i: it must be absent
    m = mass.astype(np.float64)
    d = pos[:, None, :] - pos[None, :, :]
    r = np.sqrt((d * d).sum(-1) + 0.05 ** 2)
    full = -(m[None, :] / r).sum(1)
    np.testing.assert_allclose(pot, full + m / 0.05, rtol=1e-12)


def test_direct_momentum_conservation():
    # Newton's third law: sum_i m_i a_i = 0 for a pairwise-antisymmetric force
    pos, mass = ic.hernquist(4000, 12)
    acc, _ = oracle.direct(pos, mass, 0.01)
    m = mass.astype(np.float64)[:, None]
    tot = np.abs((m * acc).sum(0))
    scale = np.abs(m * acc).sum(0)
    assert np.all(tot <= 1e-13 * scale)


def test_direct_plummer_analytic():
    # Plummer model, G = M = a = 1: phi(r) = -1/sqrt(r^2+1),
    # a_r = -r/(r^2+1)^(3/2), W = (1/2) sum m phi = -3 pi / 32.
    n = 16384
    pos, mass = ic.plummer(n, 13)
    acc, pot = oracle.direct(pos, mass, 0.005)
    r = np.linalg.norm(pos, axis=1)
    ar = (acc * pos).sum(1) / r
    edges = np.array([0.1, 0.3, 0.6, 1.0, 1.5, 2.5, 5.0])
    for lo, hi in zip(edges[:-1], edges[1:]):
        sel = (r >= lo) & (r < hi)
        rm = r[sel]
        np.testing.assert_allclose(pot[sel].mean(), (-1.0 / np.sqrt(rm * rm + 1)).mean(), rtol=0.02)
        if lo >= 0.3:  # the innermost shell holds too few particles for a_r
            np.testing.assert_allclose(ar[sel].mean(), (-rm / (rm * rm + 1) ** 1.5).mean(), rtol=0.06)
    w = 0.5 * float((mass.astype(np.float64) * pot).sum())
    assert abs(w - (-3 * math.pi / 32)) < 0.03 * 3 * math.pi / 32


def test_direct_hernquist_analytic():
    # Hernquist, truncated at rt = 100 a with M(rt) = 1: inside rt
    # phi(r) = -M_inf/(r + a) + M_inf a/(rt + a)^2, M_inf = ((rt + a)/rt)^2.
    n = 16384
    pos, mass = ic.hernquist(n, 14)
    _, pot = oracle.direct(pos, mass, 0.005)
    r = np.linalg.norm(pos, axis=1)
    minf = (101.0 / 100.0) ** 2
    for lo, hi in [(0.1, 0.3), (0.3, 1.0), (1.0, 3.0), (3.0, 10.0), (10.0, 50.0)]:
        sel = (r >= lo) & (r < hi)
        rm = r[sel]
        ref = (-minf / (rm + 1.0) + minf / 101.0 ** 2).mean()
        np.testing.assert_allclose(pot[sel].mean(), ref, rtol=0.02)


def test_cell_field_quadrupole_on_axis():
    rows = [l for l in open(GOLDEN + "/quad_axis.txt") if l.strip() and not l.startswith("#")]
    v = np.array([float(x) for x in rows[0].split()])
    x, m, q = v[0:3], v[3], v[4:10]
    m2, com, q2, b2 = oracle.cell_moments(np.array([[0, 0, 1.0], [0, 0, -1.0]]), np.array([1.0, 1.0]))
    assert m2 == m and b2 == 2.0
    np.testing.assert_allclose(com, 0, atol=1e-15)
    np.testing.assert_allclose(q2, q, atol=1e-14)
    acc, pot = oracle.cell_field(x, m, com, q, b2, True, 1e-9)
    np.testing.assert_allclose(acc, v[10:13], atol=1e-12)
    assert abs(pot - v[13]) < 1e-12
    acc, pot = oracle.cell_field(x, m, com, q, b2, False, 1e-9)
    np.testing.assert_allclose(acc, v[14:17], atol=1e-12)
    assert abs(pot - v[17]) < 1e-12


def test_cell_field_softened_quadrupole_on_axis():
    # the quadrupole term is the second-order Taylor term of the softened
    # pair law: with eps comparable to the distance its B_2 eps^2 part
    # matters (hand-worked values in the fixture)
    rows = [l for l in open(GOLDEN + "/quad_axis_soft.txt") if l.strip() and not l.startswith("#")]
    v = np.array([float(x) for x in rows[0].split()])
    x, eps, m, q, b2 = v[0:3], v[3], v[4], v[5:11], v[11]
    m2, com, q2, b22 = oracle.cell_moments(np.array([[0, 0, 1.0], [0, 0, -1.0]]), np.array([1.0, 1.0]))
    assert (m2, b22) == (m, b2)
    np.testing.assert_allclose(q2, q, atol=1e-14)
    acc, pot = oracle.cell_field(x, m, com, q, b2, True, eps)
    np.testing.assert_allclose(acc, v[12:15], rtol=0, atol=1e-15)
    assert abs(pot - v[15]) < 1e-15
    acc, pot = oracle.cell_field(x, m, com, q, b2, False, eps)
    np.testing.assert_allclose(acc, v[16:19], rtol=0, atol=1e-15)
    assert abs(pot - v[19]) < 1e-15


def test_multipole_far_field_slopes():
    # Relative error of the cell field against the exact sum over the cell's
    # particles: monopole ~ (l/d)^2 (the dipole vanishes about the centre of
    # mass), quadrupole ~ (l/d)^3.
    rng = np.random.default_rng(15)
    pts = rng.uniform(-0.5, 0.5, (25, 3))
    ms = rng.uniform(0.5, 1.5, 25)
    m, com, q, b2 = oracle.cell_moments(pts, ms)
    u = np.array([0.48, -0.6, 0.64])
    u /= np.linalg.norm(u)
    ds = np.array([8.0, 16.0, 32.0, 64.0, 128.0])
    err = {0: [], 1: []}
    for d in ds:
        x = com + d * u
        allp = np.vstack([pts, x])
        allm = np.concatenate([ms, [0.0]])
        ex_a, ex_p = oracle.direct(allp, allm, 1e-9, targets=[25])
        for quad in (0, 1):
            a, p = oracle.cell_field(x, m, com, q, b2, quad, 1e-9)
            err[quad].append(np.linalg.norm(a - ex_a[0]) / np.linalg.norm(ex_a[0]))
    s0 = np.polyfit(np.log(ds), np.log(err[0]), 1)[0]
    s1 = np.polyfit(np.log(ds), np.log(err[1]), 1)[0]
    assert abs(s0 + 2) < 0.15, s0
    assert abs(s1 + 3) < 0.15, s1
    assert all(e1 < e0 for e0, e1 in zip(err[0], err[1]))


@pytest.mark.parametrize("eps_over_d", [0.5, 2.0])
def test_softened_multipole_far_field_slopes(eps_over_d):
    # The same with Plummer softening that grows with the distance (eps =
    # c d): the expansion parameter is the cell size over sqrt(d^2 + eps^2),
    # so the second-order term must leave a third-order error (slope -3) on
    # the acceleration and the potential; a quadrupole without its B_2 eps^2
    # part leaves a second-order one.
    rng = np.random.default_rng(25)
    pts = rng.uniform(-0.5, 0.5, (25, 3))
    ms = rng.uniform(0.5, 1.5, 25)
    m, com, q, b2 = oracle.cell_moments(pts, ms)
    u = np.array([0.48, -0.6, 0.64])
    u /= np.linalg.norm(u)
    ds = np.array([8.0, 16.0, 32.0, 64.0, 128.0])
    ea, ep = [], []
    for d in ds:
        x = com + d * u
        eps = eps_over_d * d
        allp = np.vstack([pts, x])
        allm = np.concatenate([ms, [0.0]])
        ex_a, ex_p = oracle.direct(allp, allm, eps, targets=[25])
        a, p = oracle.cell_field(x, m, com, q, b2, True, eps)
        ea.append(np.linalg.norm(a - ex_a[0]) / np.linalg.norm(ex_a[0]))
        ep.append(abs(p - ex_p[0]) / abs(ex_p[0]))
    sa = np.polyfit(np.log(ds), np.log(ea), 1)[0]
    sp = np.polyfit(np.log(ds), np.log(ep), 1)[0]
    assert abs(sa + 3) < 0.15, sa
    assert abs(sp + 3) < 0.15, sp


def test_group_mac_hand_worked_cases():
    # threshold with s (just above, just below, exact tie), the cube-overlap
    # clause (overlapping, touching, clear) and theta = 0; the geometry of
    # each case is worked out in the fixture's comments
    rows = np.loadtxt(GOLDEN + "/group_mac.txt", ndmin=2)
    assert rows.shape == (7, 15)
    for r in rows:
        got = oracle.group_mac(r[0:3], r[3], r[4:7], r[7:10], r[10:13], r[13])
        assert got == bool(r[14]), r


def test_tree_quadrupole_with_large_softening():
    # the batch configuration's regime (eps a sizeable fraction of the scale
    # radius): the softened quadrupole must still beat the monopole clearly
    pos, mass = ic.plummer(3000, 26)
    eps = 4.0 * 3000 ** (-1.0 / 3.0)
    t = oracle.Tree(pos, mass, 8, 64)
    ad, pd = oracle.direct(pos, mass, eps)
    e = {}
    for quad in (False, True):
        r = t.eval(0.5, eps, use_quad=quad)
        e[quad] = oracle.errors(r["acc"], r["pot"], ad, pd)["acc_rms"]
    assert e[True] < 0.3 * e[False], e


@pytest.mark.parametrize("n,leaf,ncrit", [(1, 8, 64), (7, 8, 64), (200, 1, 4), (4096, 8, 64)])
def test_tree_theta0_is_direct_sum(n, leaf, ncrit):
    pos, mass = ic.plummer(n, 16)
    t = oracle.Tree(pos, mass, leaf, ncrit)
    r = t.eval(0.0, 0.01, use_quad=True)
    a, p = oracle.direct(pos, mass, 0.01)
    np.testing.assert_allclose(r["acc"], a, rtol=0, atol=1e-13 * np.abs(a).max())
    np.testing.assert_allclose(r["pot"], p, rtol=1e-13)
    assert r["n_cell"].sum() == 0
    assert np.all(r["n_part"] == n)
    assert r["count"].sum() == n


def test_tree_groups_partition_and_list_mass():
    pos, mass = ic.hernquist(20000, 17)
    t = oracle.Tree(pos, mass, 8, 64)
    r = t.eval(0.6, 1e-3, use_quad=True)
    assert r["count"].sum() == 20000
    assert len(np.unique(r["key"])) == t.n_groups
    assert r["count"].max() <= 64
    # every group's list covers the whole mass exactly once
    np.testing.assert_allclose(r["mass"], mass.astype(np.float64).sum(), rtol=1e-12)
    assert np.all(np.isfinite(r["acc"]))


def test_tree_features_hand_worked_two_clusters():
    # Two clusters of four: A (unit masses) at the corners 0, e x, e y, e z
    # and B (masses 2) at (100, 10, 10) + 2 {0, x, y, z}, e = 0.02.  The root
    # cube is centred on the bounding box, side S = 102 (1 + 1e-12); its
    # first split puts A in octant 0 and B in octant 7, two leaves of four
    # that are the two groups (n_crit = 4).  For group A the walk opens the
    # root and its own leaf (4 particle entries); leaf B, side l = S/2 and
    # centre lo + 3S/4, is accepted at theta = 1 (d > l + s) and opened at
    # theta = 0.5 (d < 2l + s), where its particles become entries.  The
    # softening (eps = 1) keeps A's own pull at its centre finite and large
    # against B's, so that every entry's share of it counts.
    e, eps = 0.02, 1.0
    a_pos = np.array([[0, 0, 0], [e, 0, 0], [0, e, 0], [0, 0, e]], float)
    b_pos = np.array([100.0, 10.0, 10.0]) + 2.0 * np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    pos = np.vstack([a_pos, b_pos])
    mass = np.array([1.0] * 4 + [2.0] * 4)
    t = oracle.Tree(pos, mass, 4, 4)
    assert t.n_groups == 2
    S = 102.0 * (1 + 1e-12)   # the largest extent, x: 0 .. 102
    lo = 0.5 * (pos.min(0) + pos.max(0)) - 0.5 * S
    l, gc_b = S / 2, lo + 0.75 * S
    com_b = b_pos.mean(0)
    box_lo, box_hi = a_pos.min(0), a_pos.max(0)
    d = np.linalg.norm(np.maximum(0.0, np.maximum(box_lo - com_b, com_b - box_hi)))
    s = np.linalg.norm(com_b - gc_b)
    assert l + s < d < 2 * l + s
    c = 0.5 * (box_lo + box_hi)
    h = 0.5 * np.linalg.norm(box_hi - box_lo)
    b2 = (2.0 * ((b_pos - com_b) ** 2).sum(1)).sum()       # 18
    bmax = np.sqrt(((b_pos - com_b) ** 2).sum(1)).max()     # sqrt(2.75)
    assert abs(b2 - 18.0) < 1e-12 and abs(bmax - math.sqrt(2.75)) < 1e-12
    xs, ms = np.vstack([com_b, a_pos]), np.array([8.0, 1.0, 1.0, 1.0, 1.0])
    r = xs - c
    s2 = (r * r).sum(1) + eps * eps
    pull = np.linalg.norm((ms[:, None] * r / (s2 * np.sqrt(s2))[:, None]).sum(0))
    key, f = t.features(1.0, eps)
    a = int(np.flatnonzero(key == 0)[0])
    want = [math.log2(5), math.log10(d / l), math.log10(h / eps), 8.0 / 12.0, math.log10(b2 * bmax / d ** 5 / pull)]
    assert want[4] > -11.0   # above the estimate's floor
    np.testing.assert_allclose(f[a], want, rtol=0, atol=1e-10)
    # theta = 0.5: no cell in A's list; the sentinels of the cell statistics
    key, f = t.features(0.5, eps)
    a = int(np.flatnonzero(key == 0)[0])
    np.testing.assert_allclose(f[a], [3.0, 3.0, math.log10(h / eps), 0.0, -12.0], rtol=0, atol=1e-12)
    # groups smaller than 1e-3 eps: their radius is clamped to 1e-3 eps
    key, f = t.features(1.0, 1e4)
    np.testing.assert_array_equal(f[:, 2], [-3.0, -3.0])


def test_tree_converges_as_theta_to_zero():
    pos, mass = ic.plummer(8192, 18)
    a, p = oracle.direct(pos, mass, 0.01)
    t = oracle.Tree(pos, mass, 8, 64)
    for quad in (False, True):
        prev = None
        for th in (0.9, 0.7, 0.5, 0.3, 0.1):
            e = oracle.errors(**dict(zip(("acc", "pot"), (lambda r: (r["acc"], r["pot"]))(t.eval(th, 0.01, quad)))),
                              acc_ref=a, pot_ref=p)["acc_rms"]
            if prev is not None:
                assert e < prev
            prev = e
        assert prev < (2e-5 if quad else 2e-4)
    # at equal theta the quadrupole beats the monopole
    em = oracle.errors(*(lambda r: (r["acc"], r["pot"]))(t.eval(0.5, 0.01, False)), a, p)["acc_rms"]
    eq = oracle.errors(*(lambda r: (r["acc"], r["pot"]))(t.eval(0.5, 0.01, True)), a, p)["acc_rms"]
    assert eq < 0.5 * em


def test_tree_coincident_particles_over_ncrit():
    # more than n_crit identical positions land in one maximum-depth leaf,
    # which is cut into chunks of n_crit
    pos = np.zeros((100, 3))
    pos[50:] = 1.0
    mass = np.full(100, 0.01)
    t = oracle.Tree(pos, mass, 8, 16)
    r = t.eval(0.5, 0.1)
    assert r["count"].sum() == 100 and r["count"].max() <= 16
    a, p = oracle.direct(pos, mass, 0.1)
    np.testing.assert_allclose(r["pot"], p, rtol=1e-12)


def test_tree_per_group_theta():
    pos, mass = ic.plummer(4096, 19)
    t = oracle.Tree(pos, mass, 8, 64)
    r5 = t.eval(0.5, 0.01)
    tbk = np.full(4096, 0.5)
    r = t.eval(0.9, 0.01, theta_by_key=tbk)
    np.testing.assert_array_equal(r["acc"], r5["acc"])
    tbk[r5["key"][::2]] = 0.0
    r = t.eval(0.5, 0.01, theta_by_key=tbk)
    assert np.all(r["n_cell"][::2] == 0) and np.all(r["n_part"][::2] == 4096)


# ---------------------------------------------------------------------------
# perceptron oracle

# ---- Salmon-Warren absolute MAC (Section II-B, Eq. SW_MAC, Eq. B2) ----------


@pytest.mark.parametrize("m,L,delta", [(1.0, 1.0, 0.01), (0.3, 2.0, 1e-4), (2.0, 0.5, 10.0), (1.0, 1.0, 1e-8)])
def test_sw_radius_two_particle_example(m, L, delta):
    """The paper's worked example: two particles of mass m a distance L apart
    have b_max = L/2 and B_2 = m L^2 / 2, so r_b = L/4 + sqrt(L^2/16 +
    sqrt(3 m L^2 / (2 delta))) (the printed sqrt(L/16) read as sqrt(L^2/16),
    which Eq. SW_MAC gives for b_max = L/2)."""
    pos = np.array([[0.1, -0.2, 0.3], [0.1 + L, -0.2, 0.3]])
    b2, bmax, rb = oracle.sw_radius(pos, np.array([m, m]), delta)
    assert b2 == pytest.approx(m * L * L / 2, rel=1e-14)
    assert bmax == pytest.approx(L / 2, rel=1e-14)
    assert rb == pytest.approx(L / 4 + math.sqrt(L * L / 16 + math.sqrt(3 * m * L * L / (2 * delta))), rel=1e-14)


def test_sw_radius_limits_and_mass_limit():
    rng = np.random.default_rng(5)
    pos = rng.normal(size=(40, 3))
    mass = rng.uniform(0.5, 1.5, 40)
    b2, bmax, rb_big = oracle.sw_radius(pos, mass, 1e30)
    # large delta: r_b -> b_max (the b_max MAC); small delta: r_b ~ delta^(-1/4)
    assert rb_big == pytest.approx(bmax, rel=1e-6)
    r1 = oracle.sw_radius(pos, mass, 1e-16)[2]
    r2 = oracle.sw_radius(pos, mass, 1e-16 / 16)[2]
    assert r2 / r1 == pytest.approx(2.0, rel=1e-3)
    # parallel-axis identity: B_2 = sum m |x|^2 - M |x_cm|^2
    M = mass.sum()
    xcm = (mass[:, None] * pos).sum(0) / M
    assert b2 == pytest.approx((mass * (pos ** 2).sum(1)).sum() - M * (xcm ** 2).sum(), rel=1e-12)
    # a cell heavier than m_limit gets r_b = 2 S_root
    assert oracle.sw_radius(pos, mass, 1e-3, m_limit=0.5 * M, s_root=7.0)[2] == 14.0
    assert oracle.sw_radius(pos, mass, 1e-3, m_limit=2.0 * M, s_root=7.0)[2] == oracle.sw_radius(pos, mass, 1e-3)[2]


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sw_monopole_error_within_delta(seed):
    """r_b is where the monopole error bound 3 B_2 / (d^2 (d - b_max)^2)
    equals delta: every point farther than r_b from the centre of mass sees
    the monopole within delta of the exact (unsoftened) acceleration."""
    rng = np.random.default_rng(seed)
    n = 30 if seed < 3 else 2
    pos = rng.uniform(-0.5, 0.5, size=(n, 3)) * (1.0 if seed < 3 else np.array([1.0, 0.0, 0.0]))
    mass = rng.uniform(0.1, 1.0, n)
    m, com, q, _ = oracle.cell_moments(pos, mass)
    worst = 0.0
    for delta in (1e-1, 1e-3, 1e-5):
        b2, bmax, rb = oracle.sw_radius(pos, mass, delta)
        dirs = rng.normal(size=(200, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        if seed == 3:
            dirs[:20] = [1.0, 0.0, 0.0]   # on the axis of the pair: the tight direction
        d = rb * (1.0 + 1e-9 + rng.uniform(0, 1, 200) ** 2)
        tgt = com + dirs * d[:, None]
        allp = np.vstack([pos, tgt])
        allm = np.concatenate([mass, np.zeros(len(tgt))])
        ad, _ = oracle.direct(allp, allm, 1e-12, targets=np.arange(n, n + len(tgt)))
        for k in range(len(tgt)):
            am, _ = oracle.cell_field(tgt[k], m, com, q, 0.0, False, 1e-12)
            err = np.linalg.norm(am - ad[k])
            assert err <= delta * (1 + 1e-9), (delta, k, err)
            worst = max(worst, err / delta)
    # the bound is not vacuous: nearly reached on the axis of a pair
    assert worst > (0.5 if seed == 3 else 0.05)


def test_sw_tree_error_bound_and_cost():
    """Monopole tree with the absolute MAC: each accepted cell errs by at most
    delta, so a particle's error is at most delta times its group's cell
    entries; the cost grows and the error falls as delta shrinks; a mass
    limit below every cell's mass accepts nothing (the direct sum)."""
    pos, mass = ic.plummer(3000, 31)
    mass = mass.astype(np.float64)
    ad, _ = oracle.direct(pos, mass, 1e-9)
    t = oracle.Tree(pos, mass, 8, 32)
    inter, rms = [], []
    for delta in (1e-2, 1e-3, 1e-4):
        r = t.eval(0.0, 1e-9, use_quad=False, mac="sw", delta=delta)
        err = np.linalg.norm(r["acc"] - ad, axis=1)
        assert np.all(err <= delta * r["n_cell"].max() * (1 + 1e-9))
        inter.append(r["interactions"])
        rms.append(float(np.sqrt(np.mean((err / np.linalg.norm(ad, axis=1)) ** 2))))
        assert r["n_cell"].sum() > 0
    assert inter[0] < inter[1] < inter[2]
    assert rms[0] > rms[1] > rms[2]
    r = t.eval(0.0, 0.01, use_quad=True, mac="sw", delta=1e-3, m_limit=0.5 * mass.min())
    assert np.all(r["n_cell"] == 0) and r["interactions"] == 3000 * 3000
    a2, p2 = oracle.direct(pos, mass, 0.01)
    np.testing.assert_allclose(r["acc"], a2, rtol=1e-10, atol=1e-12)


# ---- SPH sums (Section II, Bounding Radius for SPH; Eq. SPH_SUM, SPH_RAD) ----


def test_sph_kernel_shape_and_normalisation():
    integrate = pytest.importorskip("scipy.integrate")
    for h in (0.3, 1.0, 2.5):
        c = 8.0 / (math.pi * h ** 3)
        assert oracle.sph_kernel(0.0, h) == pytest.approx(c, rel=1e-15)
        assert oracle.sph_kernel(h / 2, h) == pytest.approx(c / 4, rel=1e-15)
        assert oracle.sph_kernel(h, h) == 0.0 and oracle.sph_kernel(1.5 * h, h) == 0.0
        # unit volume integral; value and slope continuous at q = 1/2
        vol = integrate.quad(lambda r: 4 * math.pi * r * r * oracle.sph_kernel(r, h), 0, h, points=[h / 2])[0]
        assert vol == pytest.approx(1.0, abs=1e-10)
        e = 1e-7 * h
        left = (oracle.sph_kernel(h / 2 - e, h) - oracle.sph_kernel(h / 2 - 2 * e, h)) / e
        right = (oracle.sph_kernel(h / 2 + 2 * e, h) - oracle.sph_kernel(h / 2 + e, h)) / e
        assert left == pytest.approx(right, rel=1e-4)
        assert left == pytest.approx(c * -1.5 / h, rel=1e-4)


def test_sph_density_closed_forms():
    # two particles: rho_1 = m_1 W(0, h_1) + m_2 W(d, h_2) (scatter form)
    pos = np.array([[0.0, 0.0, 0.0], [0.3, 0.4, 0.0]])
    m = np.array([2.0, 3.0])
    h = np.array([0.2, 0.8])
    rho = oracle.sph_density(pos, m, h)
    assert rho[0] == pytest.approx(2.0 * oracle.sph_kernel(0, 0.2) + 3.0 * oracle.sph_kernel(0.5, 0.8), rel=1e-15)
    assert rho[1] == pytest.approx(3.0 * oracle.sph_kernel(0, 0.8), rel=1e-15)   # 0.5 > h_1 = 0.2
    # a cubic lattice of unit masses with spacing a: rho = 1 / a^3 inside
    k, a = 16, 1.0 / 16
    g = (np.arange(k) + 0.5) * a
    pos = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    inner = np.nonzero(np.all(np.abs(pos - 0.5) < 0.2, axis=1))[0]
    for f in (2.0, 2.5, 3.0):
        rho = oracle.sph_density(pos, np.ones(len(pos)), np.full(len(pos), f * a), targets=inner)
        assert np.all(np.abs(rho * a ** 3 - 1.0) < 5e-3)


@pytest.mark.parametrize("model,n,leaf,ncrit", [("plummer", 4000, 8, 32), ("hernquist", 5000, 1, 64)])
def test_sph_tree_density_is_the_direct_sum(model, n, leaf, ncrit):
    """The walk only skips cells that hold no neighbour (Eq. SPH_RAD), so the
    tree density is the direct sum up to summation order, from far fewer
    pairs."""
    pos, mass = ic.make(model, n, 36)
    mass = mass.astype(np.float64)
    h = 0.02 + 0.3 * np.random.default_rng(1).random(n) * np.minimum(1.0, np.linalg.norm(pos, axis=1))
    r = oracle.Tree(pos, mass, leaf, ncrit).sph_density(h)
    d = oracle.sph_density(pos, mass, h)
    np.testing.assert_allclose(r["rho"], d, rtol=1e-12, atol=0)
    assert r["pairs"] < 0.2 * n * n


from oracle import mlp as omlp  # noqa: E402


def test_mlp_layout_and_bias_only_network():
    assert omlp.NP == 1313
    w = np.zeros(omlp.NP)
    w[-1] = 0.75  # b3 only: y = b3 for every row
    x = np.random.default_rng(1).normal(size=(10, 6))
    np.testing.assert_array_equal(omlp.forward(w, x), 0.75)
    # one hidden path: y = w3[0] tanh(W2[0,0] tanh(W1[0,2] x2))
    w = np.zeros(omlp.NP)
    W1, b1, W2, b2, w3, b3 = [a for a in omlp.unpack(np.arange(omlp.NP, dtype=float))]
    w[2] = 0.5                      # W1[0][2]
    w[192 + 32] = 2.0               # W2[0][0]
    w[192 + 32 + 1024 + 32] = 3.0   # w3[0]
    y = omlp.forward(w, x)
    np.testing.assert_allclose(y, 3.0 * np.tanh(2.0 * np.tanh(0.5 * x[:, 2])), rtol=1e-15)


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    w = rng.normal(scale=0.4, size=omlp.NP)
    x = rng.normal(size=(40, 6))
    t = rng.normal(size=40)
    g = omlp.grad(w, x, t)
    h = 1e-6
    idx = np.concatenate([rng.choice(omlp.NP, 60, replace=False), [0, 191, 192, 1311, 1312]])
    for k in idx:
        e = np.zeros(omlp.NP)
        e[k] = h
        fd = (omlp.loss(w + e, x, t) - omlp.loss(w - e, x, t)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), (k, fd, g[k])


def test_adam_first_step_and_bf16_rounding():
    # first Adam step moves every weight by lr * sign(g) (bias correction)
    g = np.array([0.3, -2.0, 1e-3])
    w, m, v = omlp.adam(np.zeros(3), np.zeros(3), np.zeros(3), g, 1, lr=0.01, eps=0.0)
    np.testing.assert_allclose(w, -0.01 * np.sign(g), rtol=1e-12)
    # bf16: 8 significand bits, ties to even
    np.testing.assert_array_equal(omlp.bf16_round([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -3.0]),
                                  [1.0, 1.0, 1.0 + 2 ** -6, -3.0])


def test_choose_theta_hand_built_tables():
    # the angle choice on hand-built prediction tables (cases described in
    # the fixture): largest passing angle, ties pass, none -> grid[0],
    # non-finite -> fallback, per-group targets
    from oracle import mlp as om
    rows = np.genfromtxt(GOLDEN + "/select_theta.txt", comments="#")
    grid = [0.3, 0.4, 0.5, 0.6]
    got = om.choose_theta(rows[:, 0:4], grid, rows[:, 4], 0.45)
    np.testing.assert_array_equal(got, rows[:, 5])
    # one target for every group gives the same answer where it is the same
    same = rows[:, 4] == -3.0
    np.testing.assert_array_equal(om.choose_theta(rows[same, 0:4], grid, -3.0, 0.45), rows[same, 5])


def test_select_theta_wires_the_network_to_the_choice():
    # a bias-only network predicts the same value for every row: all angles
    # pass below the target, none above it
    from oracle import mlp as om
    w = np.zeros(om.NP)
    feats = np.random.default_rng(40).normal(size=(5, 4, om.NI))
    grid = [0.3, 0.4, 0.5, 0.6]
    w[-1] = -3.2
    th, y = om.select_theta(w, feats, grid, -3.0, 0.45)
    assert np.all(y == -3.2) and np.all(th == 0.6)
    w[-1] = -2.8
    th, _ = om.select_theta(w, feats, grid, -3.0, 0.45)
    assert np.all(th == 0.3)


def test_budget_targets_closed_forms():
    from oracle import mlp as om
    # equal predictions and lists: every group aims at the RMS target itself
    t = om.budget_targets([-3.0, -3.0, -3.0], [10, 10, 10], [5, 7, 9], 1e-3, 1.0 / 3, 1.0 / 3)
    np.testing.assert_allclose(t, -3.0, atol=1e-12)
    # two groups of equal size, predictions 10^-2 and 10^-4 at theta0, equal
    # lists, alpha = 1/2: weights 10^-1 and 10^-2; lambda = T / sqrt((10^-2
    # + 10^-4) / 2), worked by hand for T = 1e-3
    t = om.budget_targets([-2.0, -4.0], [8, 8], [10, 10], 1e-3, 0.5, 0.0)
    lam = 1e-3 / np.sqrt((1e-2 + 1e-4) / 2)
    np.testing.assert_allclose(t, np.log10([lam * 0.1, lam * 0.01]), rtol=0, atol=1e-12)
    # the list-length exponent: equal predictions, lists of 2^10 and 2^13
    # with beta = 1/3 give targets in the ratio 2
    t = om.budget_targets([-3.0, -3.0], [10, 13], [1, 1], 1e-3, 1.0 / 3, 1.0 / 3)
    np.testing.assert_allclose(t[1] - t[0], np.log10(2.0), atol=1e-12)
    # always: the particle-weighted RMS of the targets is the RMS target
    rng = np.random.default_rng(41)
    y0, ll, n = rng.normal(-3, 1, 50), rng.uniform(5, 14, 50), rng.integers(1, 128, 50)
    t = om.budget_targets(y0, ll, n, 2e-3, 1.0 / 3, 1.0 / 3)
    np.testing.assert_allclose(np.sqrt(np.sum(n * 100.0 ** t) / n.sum()), 2e-3, rtol=1e-12)


def test_learned_theta_range_and_fallback():
    # a bias-only network (prediction -3.2 everywhere): groups in range all
    # pass every angle; a statistic outside [lo, hi] or a NaN gives the
    # fallback, and the out-of-range groups do not enter lambda
    from oracle import mlp as om
    w = np.zeros(om.NP)
    w[-1] = -3.2
    feats = np.array([[10.0, 0.5, 1.0, 0.4, -1.0], [11.0, 0.5, 1.0, 0.4, -1.0], [30.0, 0.5, 1.0, 0.4, -1.0],
                      [10.0, np.nan, 1.0, 0.4, -1.0]])
    lo, hi = np.full(5, -20.0), np.full(5, 20.0)
    grid = [0.3, 0.5, 0.7]
    th, tg = om.learned_theta(w, np.zeros(6), np.ones(6), lo, hi, feats, [4, 4, 4, 4], grid, 0.5, 1e-3, 1.0, 1.0 / 3,
                              0.0, 0.45)
    np.testing.assert_array_equal(th, [0.7, 0.7, 0.45, 0.45])
    np.testing.assert_allclose(tg[:2], -3.0, atol=1e-12)
    assert np.all(np.isnan(tg[2:]))


def test_error_statistics_hand_worked():
    # two targets: reference accelerations (3, 4, 0) and (0, 0, 2); the first
    # is off by (0.03, 0, 0) (relative 0.03 / 5 = 0.006), the second exact;
    # potentials -2 and -4, the second off by 0.04 (relative 0.01)
    ref = np.array([[3.0, 4.0, 0.0], [0.0, 0.0, 2.0]])
    acc = ref + np.array([[0.03, 0.0, 0.0], [0.0, 0.0, 0.0]])
    e = oracle.errors(acc, np.array([-2.0, -4.04]), ref, np.array([-2.0, -4.0]))
    assert abs(e["acc_max"] - 0.006) < 1e-15 and abs(e["acc_mean"] - 0.003) < 1e-15
    assert abs(e["acc_rms"] - 0.006 / np.sqrt(2)) < 1e-15
    assert abs(e["pot_max"] - 0.01) < 1e-15 and abs(e["pot_rms"] - 0.01 / np.sqrt(2)) < 1e-15
