"""FP64 CPU oracle for softened gravity (direct sum, octree, MLP).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only users.  Nothing here is shared
with the GPU path (the two sides read the same seeded inputs and nothing else).

* ``direct``      Plummer-softened direct sum, G = 1, j != i (Section II,
                  particle-particle interaction; pair law is a reading, the
                  paper does not print it).
* ``Tree``        octree, groups, group walk with the opening-angle MAC or
                  the Salmon-Warren absolute MAC (Section II-B, Eq. SW_MAC),
                  and the force over each group's walk (Sections II, III-B,
                  III-C, III-D), monopole or quadrupole cells.
* ``sw_radius``   B_2 (Eq. B2), b_max and r_b (Eq. SW_MAC) of one particle set.
* ``sph_kernel`` / ``sph_density``  the SPH kernel W and the density
                  rho_i = sum_j m_j W(|x_i - x_j|, h_j) (Eq. SPH_SUM) by direct
                  summation; ``Tree.sph_density`` through the group walk with
                  the bounding radius of Eq. SPH_RAD.
* ``cell_moments`` / ``cell_field``  the multipole of one particle set and
                  its field at a point.
* ``group_mac``   the opening-angle acceptance test of the group walk.
* ``Tree.features``  the five list statistics of each group's walk that feed
                  the learned opening angle (a reading of this project; the
                  paper's accuracy control is Delta, Section II-B).
* ``errors``      relative force error statistics against a reference.

The C part is compiled by ``__graft_entry__.build()`` (gcc, -O2 -fopenmp
-ffp-contract=off) into ``oracle/liboracle.so``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lib = None

_i64 = ctypes.c_int64
_dp = ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)


def compile_oracle(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (plain gcc; no GPU involved)."""
    src = os.path.join(_HERE, "oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c99", src, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        compile_oracle()
        lib = ctypes.CDLL(_SO)
        lib.oracle_direct.argtypes = [_i64, _dp, _dp, _i64, _lp, ctypes.c_double, _dp, _dp]
        lib.oracle_direct.restype = ctypes.c_int
        lib.oracle_cell_moments.argtypes = [_dp, _dp, _i64, _dp, _dp, _dp, _dp]
        lib.oracle_cell_moments.restype = ctypes.c_int
        lib.oracle_cell_field.argtypes = [_dp, ctypes.c_double, _dp, _dp, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_double, _dp, _dp]
        lib.oracle_group_mac.argtypes = [_dp, ctypes.c_double, _dp, _dp, _dp, ctypes.c_double,
                                         ctypes.POINTER(ctypes.c_int)]
        lib.oracle_group_mac.restype = ctypes.c_int
        lib.oracle_cell_field.restype = ctypes.c_int
        lib.oracle_tree_new.argtypes = [_i64, _dp, _dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_tree_new.restype = ctypes.c_void_p
        lib.oracle_tree_free.argtypes = [ctypes.c_void_p]
        lib.oracle_tree_free.restype = None
        lib.oracle_tree_n_groups.argtypes = [ctypes.c_void_p]
        lib.oracle_tree_n_groups.restype = _i64
        lib.oracle_tree_n_cells.argtypes = [ctypes.c_void_p]
        lib.oracle_tree_n_cells.restype = _i64
        lib.oracle_tree_eval.argtypes = [ctypes.c_void_p, ctypes.c_double, _dp, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_double, ctypes.c_double, ctypes.c_int, _i64, _lp, _i64, _dp,
                                         _dp, _lp, _lp, _lp, _lp, _dp, _lp]
        lib.oracle_tree_eval.restype = ctypes.c_int
        lib.oracle_sw_radius.argtypes = [_dp, _dp, _i64, ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_sw_radius.restype = ctypes.c_int
        lib.oracle_sph_kernel.argtypes = [ctypes.c_double, ctypes.c_double, _dp]
        lib.oracle_sph_kernel.restype = ctypes.c_int
        lib.oracle_sph_density_direct.argtypes = [_i64, _dp, _dp, _dp, _i64, _lp, _dp]
        lib.oracle_sph_density_direct.restype = ctypes.c_int
        lib.oracle_tree_sph_density.argtypes = [ctypes.c_void_p, _dp, _dp, _lp, _lp, _lp]
        lib.oracle_tree_sph_density.restype = ctypes.c_int
        lib.oracle_tree_features.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _lp, _dp]
        lib.oracle_tree_features.restype = ctypes.c_int
        _lib = lib
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _l(a):
    return a.ctypes.data_as(_lp)


def direct(pos, mass, eps, targets=None):
    """Direct sum.  pos [n][3], mass [n] (any float type, used as FP64).

    Returns (acc [k][3], pot [k]) for the target indices (default: all)."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    n = pos.shape[0]
    tgt = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    acc = np.zeros((tgt.shape[0], 3))
    pot = np.zeros(tgt.shape[0])
    rc = lib.oracle_direct(n, _d(pos), _d(mass), tgt.shape[0], _l(tgt), float(eps), _d(acc), _d(pot))
    if rc != 0:
        raise ValueError("oracle_direct: bad arguments")
    return acc, pot


def cell_moments(pos, mass):
    """(mass, com[3], q[6], b2) with q = (Qxx, Qyy, Qzz, Qxy, Qxz, Qyz) the
    traceless quadrupole about the com and b2 = sum m |x - com|^2."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    m = np.zeros(1)
    com = np.zeros(3)
    q = np.zeros(6)
    b2 = np.zeros(1)
    if lib.oracle_cell_moments(_d(pos), _d(mass), pos.shape[0], _d(m), _d(com), _d(q), _d(b2)) != 0:
        raise ValueError("empty cell")
    return float(m[0]), com, q, float(b2[0])


def sw_radius(pos, mass, delta, m_limit=0.0, s_root=1.0):
    """(B_2, b_max, r_b) of one particle set for the absolute MAC."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    out = np.zeros(3)
    if lib.oracle_sw_radius(_d(pos), _d(mass), pos.shape[0], float(delta), float(m_limit), float(s_root),
                            _d(out)) != 0:
        raise ValueError("empty cell")
    return float(out[0]), float(out[1]), float(out[2])


def sph_kernel(r, h):
    """W(r, h) of the SPH sums (M4 cubic spline, support radius h)."""
    lib = _load()
    w = np.zeros(1)
    if lib.oracle_sph_kernel(float(r), float(h), _d(w)) != 0:
        raise ValueError("bad r or h")
    return float(w[0])


def sph_density(pos, mass, h, targets=None):
    """rho_i = sum_j m_j W(|x_i - x_j|, h_j) by direct summation."""
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    n = pos.shape[0]
    tgt = np.arange(n, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    rho = np.zeros(tgt.shape[0])
    if lib.oracle_sph_density_direct(n, _d(pos), _d(mass), _d(h), tgt.shape[0], _l(tgt), _d(rho)) != 0:
        raise ValueError("oracle_sph_density_direct: bad arguments")
    return rho


def cell_field(x, m, com, q, b2, use_quad, eps):
    """Field (acc[3], pot) at point x of a cell with the given moments
    (b2 = sum m |x - com|^2 enters the softened quadrupole term)."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.float64)
    com = np.ascontiguousarray(com, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    acc = np.zeros(3)
    pot = np.zeros(1)
    lib.oracle_cell_field(_d(x), float(m), _d(com), _d(q), float(b2), int(use_quad), float(eps), _d(acc),
                          _d(pot))
    return acc, float(pot[0])


def group_mac(cube_lo, side, com, blo, bhi, theta):
    """The tree walk's opening-angle decision for one cell (cube corner
    cube_lo, side, centre of mass com) and one group box [blo, bhi]:
    True = accept the cell, False = open it."""
    lib = _load()
    v = [np.ascontiguousarray(a, dtype=np.float64) for a in (cube_lo, com, blo, bhi)]
    out = ctypes.c_int(-1)
    if lib.oracle_group_mac(_d(v[0]), float(side), _d(v[1]), _d(v[2]), _d(v[3]), float(theta),
                            ctypes.byref(out)) != 0:
        raise ValueError("bad cell or angle")
    return bool(out.value)


class Tree:
    """Octree over one particle system (inputs are copied and kept alive)."""

    def __init__(self, pos, mass, leaf_size=8, n_crit=64):
        self._lib = _load()
        self.pos = np.ascontiguousarray(pos, dtype=np.float64)
        self.mass = np.ascontiguousarray(mass, dtype=np.float64)
        self.n = self.pos.shape[0]
        self._h = self._lib.oracle_tree_new(self.n, _d(self.pos), _d(self.mass), int(leaf_size), int(n_crit))
        if not self._h:
            raise ValueError("oracle_tree_new failed")
        self.n_groups = int(self._lib.oracle_tree_n_groups(self._h))
        self.n_cells = int(self._lib.oracle_tree_n_cells(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_tree_free(h)
            self._h = None

    def eval(self, theta, eps, use_quad=False, theta_by_key=None, group_stride=1, mac="theta", delta=0.0,
             m_limit=0.0, groups=None):
        """Tree force.  mac = "theta" (opening angle theta, or theta_by_key)
        or "sw" (absolute MAC with accuracy delta; cells heavier than m_limit
        > 0 are never accepted).  Every group is walked and every
        group_stride-th one evaluated; or, with groups (group indices), only
        those are walked and evaluated.  Returns dict with acc, pot (caller
        order; NaN for particles of skipped groups) and per-group statistics
        (zero for groups that were not walked)."""
        ng = self.n_groups
        acc = np.full((self.n, 3), np.nan)
        pot = np.full(self.n, np.nan)
        key = np.zeros(ng, np.int64)
        cnt = np.zeros(ng, np.int64)
        ncell = np.zeros(ng, np.int64)
        npart = np.zeros(ng, np.int64)
        gmass = np.zeros(ng)
        inter = np.zeros(1, np.int64)
        tbk = None
        if theta_by_key is not None:
            tbk = np.ascontiguousarray(theta_by_key, dtype=np.float64)
            assert tbk.shape[0] == self.n
        kind = {"theta": 0, "sw": 1}[mac]
        sel = None if groups is None else np.ascontiguousarray(groups, dtype=np.int64)
        rc = self._lib.oracle_tree_eval(self._h, float(theta), _d(tbk) if tbk is not None else None,
                                        kind, float(delta), float(m_limit), float(eps), int(bool(use_quad)),
                                        int(group_stride), _l(sel) if sel is not None else None,
                                        0 if sel is None else sel.shape[0], _d(acc), _d(pot), _l(key), _l(cnt),
                                        _l(ncell), _l(npart), _d(gmass), _l(inter))
        if rc != 0:
            raise ValueError("oracle_tree_eval failed (%d)" % rc)
        return dict(acc=acc, pot=pot, key=key, count=cnt, n_cell=ncell, n_part=npart,
                    mass=gmass, interactions=int(inter[0]))


def _tree_sph_density(self, h):
    """Density through the group walk (Eq. SPH_RAD); returns dict with rho
    (caller order), per-group key / n_part and the pair count."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    assert h.shape == (self.n,)
    rho = np.full(self.n, np.nan)
    key = np.zeros(self.n_groups, np.int64)
    npart = np.zeros(self.n_groups, np.int64)
    pairs = np.zeros(1, np.int64)
    if self._lib.oracle_tree_sph_density(self._h, _d(h), _d(rho), _l(key), _l(npart), _l(pairs)) != 0:
        raise ValueError("oracle_tree_sph_density failed")
    return dict(rho=rho, key=key, n_part=npart, pairs=int(pairs[0]))


Tree.sph_density = _tree_sph_density


def _tree_features(self, theta, eps):
    """The five list statistics of each group's walk at opening angle theta
    (oracle_tree_features: list length, nearest cell distance over size, box
    radius over eps, cell mass fraction, truncation estimate over the net
    pull); returns (key [n_groups], feat [n_groups][5])."""
    key = np.zeros(self.n_groups, np.int64)
    feat = np.zeros((self.n_groups, 5), np.float64)
    if self._lib.oracle_tree_features(self._h, float(theta), float(eps), _l(key), _d(feat)) != 0:
        raise ValueError("oracle_tree_features failed")
    return key, feat


Tree.features = _tree_features


def errors(acc, pot, acc_ref, pot_ref):
    """Relative error statistics: delta_i = |a_i - a_ref| / |a_ref| (and the
    same for the potential); returns rms, max and mean of both."""
    acc = np.asarray(acc, np.float64)
    acc_ref = np.asarray(acc_ref, np.float64)
    da = np.linalg.norm(acc - acc_ref, axis=1) / np.linalg.norm(acc_ref, axis=1)
    dp = np.abs(np.asarray(pot, np.float64) - pot_ref) / np.abs(pot_ref)
    return dict(acc_rms=float(np.sqrt(np.mean(da * da))), acc_max=float(da.max()),
                acc_mean=float(da.mean()), pot_rms=float(np.sqrt(np.mean(dp * dp))),
                pot_max=float(dp.max()), pot_mean=float(dp.mean()))
