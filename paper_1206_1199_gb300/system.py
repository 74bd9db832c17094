"""Python front end of the C ABI: host tree/lists/plan handles, upload to
device memory (PyTorch tensors as plain buffers) and the force call.

Every step of the force computation runs in libotoo (host walk in C++,
force in CUDA); this module only moves arguments and buffers around."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _lib as L


def _params(theta, leaf_size, n_crit, use_quad, eps, theta_per_group=None):
    p = L.Params()
    p.theta = float(theta)
    p.leaf_size = int(leaf_size)
    p.n_crit = int(n_crit)
    p.use_quad = int(bool(use_quad))
    p.eps = float(eps)
    if theta_per_group is not None:
        p.theta_per_group = theta_per_group.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    return p


class Tree:
    """Host octree of one particle system (otoo_build_tree)."""

    def __init__(self, pos, mass, leaf_size=8):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        mass = np.ascontiguousarray(mass, dtype=np.float32)
        assert pos.ndim == 2 and pos.shape[1] == 3 and mass.shape == (pos.shape[0],)
        self.n = pos.shape[0]
        self.leaf_size = leaf_size
        h = ctypes.c_void_p()
        p = _params(0.5, leaf_size, 64, 0, 1.0)
        L.call("otoo_build_tree", pos.ctypes.data, mass.ctypes.data, self.n, ctypes.byref(p), ctypes.byref(h))
        self._h = h

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            L.load().otoo_tree_free(self._h)
            self._h = None

    def export(self):
        v = L.TreeView()
        L.call("otoo_tree_export", self._h, ctypes.byref(v))
        nc = v.n_cell
        return dict(n_part=v.n_part, n_cell=nc, depth=v.depth, root_lo=np.array(v.root_lo), root_side=v.root_side,
                    pos=L.view(v.pos, np.float64, (v.n_part, 3)), mass=L.view(v.mass, np.float32, (v.n_part,)),
                    perm=L.view(v.perm, np.int64, (v.n_part,)), begin=L.view(v.cell_begin, np.int64, (nc,)),
                    end=L.view(v.cell_end, np.int64, (nc,)), level=L.view(v.cell_level, np.int32, (nc,)),
                    nchild=L.view(v.cell_nchild, np.int32, (nc,)), child0=L.view(v.cell_child0, np.int64, (nc,)),
                    org=L.view(v.cell_org, np.int64, (nc, 3)), com=L.view(v.cell_com, np.float64, (nc, 3)),
                    cmass=L.view(v.cell_mass, np.float64, (nc,)), quad=L.view(v.cell_quad, np.float64, (nc, 6)))

    def lists(self, theta, n_crit, eps, use_quad=True, theta_per_group=None):
        return Lists.make(self, theta, n_crit, eps, use_quad, theta_per_group)


class Lists:
    """Groups and interaction lists (otoo_make_groups_and_lists / otoo_pack_batch)."""

    def __init__(self, handle, keep=()):
        self._h = handle
        self._keep = keep
        v = L.ListsView()
        L.call("otoo_lists_export", self._h, ctypes.byref(v))
        self.view_struct = v
        self.n_part, self.n_src, self.n_groups, self.n_list = v.n_part, v.n_src, v.n_groups, v.n_list
        self.n_sys, self.use_quad = v.n_sys, v.use_quad
        self.interactions, self.cell_interactions = v.interactions, v.cell_interactions

    @classmethod
    def make(cls, tree, theta, n_crit, eps, use_quad=True, theta_per_group=None):
        tpg = None
        if theta_per_group is not None:
            tpg = np.ascontiguousarray(theta_per_group, dtype=np.float32)
        p = _params(theta, tree.leaf_size, n_crit, use_quad, eps, tpg)
        h = ctypes.c_void_p()
        L.call("otoo_make_groups_and_lists", tree._h, ctypes.byref(p), ctypes.byref(h))
        return cls(h, keep=(tree,))

    @classmethod
    def pack(cls, lists_seq):
        arr = (ctypes.c_void_p * len(lists_seq))(*[l._h.value for l in lists_seq])
        h = ctypes.c_void_p()
        L.call("otoo_pack_batch", arr, len(lists_seq), ctypes.byref(h))
        return cls(h, keep=tuple(lists_seq))

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            L.load().otoo_lists_free(self._h)
            self._h = None

    # numpy views of the library-owned arrays (valid while self lives)
    @property
    def src(self):
        return L.view(self.view_struct.src, np.dtype(L.Src), (self.n_src,))

    @property
    def quad(self):
        return L.view(self.view_struct.quad, np.dtype(L.Quad), (self.n_src - self.n_part,))

    @property
    def groups(self):
        return L.view(self.view_struct.groups, np.dtype(L.Group), (self.n_groups,))

    @property
    def list(self):
        return L.view(self.view_struct.list, np.int32, (self.n_list,))

    @property
    def perm(self):
        return L.view(self.view_struct.perm, np.int64, (self.n_part,))

    @property
    def sys_part_off(self):
        return L.view(self.view_struct.sys_part_off, np.int64, (self.n_sys + 1,))

    def features(self, tree):
        f = np.zeros((self.n_groups, 5), np.float32)
        L.call("otoo_group_features", tree._h, self._h, f.ctypes.data)
        return f

    def plan(self, tune):
        return Plan(self, tune)


class Plan:
    """Work items (otoo_make_plan)."""

    def __init__(self, lists, tune):
        self.tune = tune
        h = ctypes.c_void_p()
        L.call("otoo_make_plan", lists._h, ctypes.byref(tune), ctypes.byref(h))
        self._h = h
        self._lists = lists
        info = L.PlanInfo()
        L.call("otoo_plan_export", h, ctypes.byref(info))
        self.info = info
        self.n_items, self.n_splits = info.n_items, info.n_splits
        self.partial_doubles, self.n_crit_max = info.partial_doubles, info.n_crit_max

    def __del__(self):
        if getattr(self, "_h", None) and self._h.value:
            L.load().otoo_plan_free(self._h)
            self._h = None

    @property
    def items(self):
        return L.view(self.info.items, np.dtype(L.Item), (self.n_items,))

    @property
    def splits(self):
        return L.view(self.info.splits, np.dtype(L.Split), (self.n_splits,))


def _to_dev(arr, device):
    import torch
    a = np.ascontiguousarray(arr)
    t = torch.from_numpy(a.view(np.uint8).reshape(-1).copy() if a.size else np.zeros(16, np.uint8))
    return t.to(device)


@dataclass
class DeviceSystem:
    """Device copies of one step's inputs plus scratch (torch uint8 buffers)."""
    lists: Lists
    plan: Plan
    bufs: dict = field(default_factory=dict)
    struct: L.DevSystem = None
    use_perm: bool = True

    @classmethod
    def upload(cls, lists, plan, device="cuda", use_perm=True):
        import torch
        b = {}
        b["src"] = _to_dev(lists.src, device)
        b["quad"] = _to_dev(lists.quad, device) if lists.use_quad and lists.n_src > lists.n_part else None
        b["groups"] = _to_dev(lists.groups, device)
        b["list"] = _to_dev(lists.list, device)
        b["items"] = _to_dev(plan.items, device)
        b["splits"] = _to_dev(plan.splits, device) if plan.n_splits else None
        b["perm"] = _to_dev(lists.perm, device) if use_perm else None
        b["partial"] = torch.empty(max(plan.partial_doubles, 1), dtype=torch.float64, device=device)
        b["counter"] = torch.zeros(4, dtype=torch.int32, device=device)
        b["split"] = torch.empty(lists.n_src * 8, dtype=torch.float32, device=device)
        s = L.DevSystem()
        s.n_part, s.n_src, s.n_list = lists.n_part, lists.n_src, lists.n_list
        s.n_groups, s.n_items, s.n_splits, s.n_crit_max = lists.n_groups, plan.n_items, plan.n_splits, plan.n_crit_max
        for k in ("src", "quad", "groups", "list", "items", "splits", "perm", "partial", "counter", "split"):
            setattr(s, k, b[k].data_ptr() if b[k] is not None else None)
        return cls(lists=lists, plan=plan, bufs=b, struct=s, use_perm=use_perm)

    def h2d_bytes(self):
        return sum(v.numel() * v.element_size() for k, v in self.bufs.items()
                   if v is not None and k not in ("partial", "counter", "split"))


def force(dev, accel=None, pot=None, precision=L.OTOO_FP32K, tune=None, stream=None, check=True):
    """otoo_force on a DeviceSystem; returns (accel [n][3], pot [n]) FP64
    tensors in caller order (tree order when the system has no perm)."""
    import torch
    n = dev.lists.n_part
    device = dev.bufs["src"].device
    if accel is None:
        accel = torch.empty((n, 3), dtype=torch.float64, device=device)
    if pot is None:
        pot = torch.empty(n, dtype=torch.float64, device=device)
    tune = tune if tune is not None else dev.plan.tune
    st = stream if stream is not None else torch.cuda.current_stream(device)
    L.call("otoo_force", ctypes.byref(dev.struct), accel.data_ptr(), pot.data_ptr(), int(precision),
           ctypes.byref(tune), ctypes.c_void_p(st.cuda_stream))
    if check:
        L.call("otoo_check_status", ctypes.byref(dev.struct), ctypes.c_void_p(st.cuda_stream))
    return accel, pot


def force_host(lists, plan, precision=L.OTOO_FP32K, tune=None, stream=None, accel=None, pot=None, view=None):
    """otoo_force_host: host arrays in, host arrays out (caller order)."""
    import torch
    n = lists.n_part
    if accel is None:
        accel = np.empty((n, 3), np.float64)
    if pot is None:
        pot = np.empty(n, np.float64)
    tune = tune if tune is not None else plan.tune
    st = stream if stream is not None else torch.cuda.current_stream()
    v = view if view is not None else lists.view_struct
    L.call("otoo_force_host", ctypes.byref(v), ctypes.byref(plan.info), L.ptr(accel), L.ptr(pot), int(precision),
           ctypes.byref(tune), ctypes.c_void_p(st.cuda_stream))
    return accel, pot


def build_system(pos, mass, theta, n_crit, eps, leaf_size=8, use_quad=True, tune=None):
    """Tree, lists and plan of one system on the host."""
    tree = Tree(pos, mass, leaf_size)
    lists = tree.lists(theta, n_crit, eps, use_quad)
    tune = tune if tune is not None else L.default_tune(max(n_crit, int(lists.groups["count"].max())))
    return tree, lists, lists.plan(tune)
