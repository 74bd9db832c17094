"""Python front end of the C ABI: host tree/lists/plan handles, upload to
device memory (PyTorch tensors as plain buffers) and the force call.

Every step of the force computation runs in libotoo (host walk in C++,
force in CUDA); this module only moves arguments and buffers around."""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import _lib as L


MAC_KINDS = {"theta": L.OTOO_MAC_THETA, "sw": L.OTOO_MAC_SW, "sph": L.OTOO_MAC_SPH}


def _params(theta, leaf_size, n_crit, use_quad, eps, theta_per_group=None, mac="theta", delta=0.0, m_limit=0.0,
            h_sph=None):
    """otoo_params; h_sph (OTOO_MAC_SPH) must be a float32 numpy array kept
    alive by the caller for the call."""
    p = L.Params()
    p.theta = float(theta)
    p.leaf_size = int(leaf_size)
    p.n_crit = int(n_crit)
    p.use_quad = int(bool(use_quad))
    p.mac = MAC_KINDS[mac]
    if h_sph is not None:
        assert h_sph.dtype == np.float32 and h_sph.flags.c_contiguous
        p.h_sph = h_sph.ctypes.data
    p.eps = float(eps)
    p.delta = float(delta)
    p.m_limit = float(m_limit)
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
                    cmass=L.view(v.cell_mass, np.float64, (nc,)), quad=L.view(v.cell_quad, np.float64, (nc, 6)),
                    b2=L.view(v.cell_b2, np.float64, (nc,)), bmax=L.view(v.cell_bmax, np.float64, (nc,)),
                    tree=self)  # the views borrow the tree's memory: keep it alive

    def lists(self, theta, n_crit, eps, use_quad=True, theta_per_group=None, mac="theta", delta=0.0, m_limit=0.0,
              h_sph=None):
        """Groups and lists; mac = "theta" (opening angle), "sw" (absolute
        MAC with accuracy delta and mass limit m_limit) or "sph" (neighbour
        lists for the radii h_sph, caller order)."""
        return Lists.make(self, theta, n_crit, eps, use_quad, theta_per_group, mac, delta, m_limit, h_sph)


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
    def make(cls, tree, theta, n_crit, eps, use_quad=True, theta_per_group=None, mac="theta", delta=0.0,
             m_limit=0.0, h_sph=None):
        tpg = None
        if theta_per_group is not None:
            tpg = np.ascontiguousarray(theta_per_group, dtype=np.float32)
        hs = None if h_sph is None else np.ascontiguousarray(h_sph, dtype=np.float32)
        p = _params(theta, tree.leaf_size, n_crit, use_quad, eps, tpg, mac, delta, m_limit, hs)
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
        s.partial_doubles = b["partial"].numel()
        s.n_groups, s.n_items, s.n_splits, s.n_crit_max = lists.n_groups, plan.n_items, plan.n_splits, plan.n_crit_max
        for k in ("src", "quad", "groups", "list", "items", "splits", "perm", "partial", "counter", "split"):
            setattr(s, k, b[k].data_ptr() if b[k] is not None else None)
        return cls(lists=lists, plan=plan, bufs=b, struct=s, use_perm=use_perm)

    @property
    def n_part(self):
        return self.lists.n_part

    @property
    def tune(self):
        return self.plan.tune

    def h2d_bytes(self):
        return sum(v.numel() * v.element_size() for k, v in self.bufs.items()
                   if v is not None and k not in ("partial", "counter", "split"))


def force(dev, accel=None, pot=None, precision=L.OTOO_FP32K, tune=None, stream=None, check=True):
    """otoo_force on a DeviceSystem; returns (accel [n][3], pot [n]) FP64
    tensors in caller order (tree order when the system has no perm)."""
    import torch
    n = dev.n_part
    device = dev.bufs["src"].device
    if accel is None:
        accel = torch.empty((n, 3), dtype=torch.float64, device=device)
    if pot is None:
        pot = torch.empty(n, dtype=torch.float64, device=device)
    tune = tune if tune is not None else dev.tune
    st = stream if stream is not None else torch.cuda.current_stream(device)
    L.call("otoo_force", ctypes.byref(dev.struct), accel.data_ptr(), pot.data_ptr(), int(precision),
           ctypes.byref(tune), ctypes.c_void_p(st.cuda_stream))
    if check:
        L.call("otoo_check_status", ctypes.byref(dev.struct), ctypes.c_void_p(st.cuda_stream))
    return accel, pot


def sph_density(dev, h, rho=None, tune=None, stream=None, check=True):
    """otoo_sph_density on a DeviceSystem or DeviceStep made from SPH lists:
    h = neighbour radii (caller order; numpy array or device tensor);
    returns rho [n] FP64 (caller order)."""
    import torch
    n = dev.n_part
    device = dev.bufs["src"].device
    if torch.is_tensor(h):
        hd = h.to(device=device, dtype=torch.float32).contiguous()
    else:
        hd = torch.from_numpy(np.ascontiguousarray(h, dtype=np.float32)).to(device)
    if rho is None:
        rho = torch.empty(n, dtype=torch.float64, device=device)
    tune = tune if tune is not None else dev.tune
    st = stream if stream is not None else torch.cuda.current_stream(device)
    L.call("otoo_sph_density", ctypes.byref(dev.struct), hd.data_ptr(), rho.data_ptr(), ctypes.byref(tune),
           ctypes.c_void_p(st.cuda_stream))
    if check:
        L.call("otoo_check_status", ctypes.byref(dev.struct), ctypes.c_void_p(st.cuda_stream))
    return rho


def _particle_sources(pos, mass, device):
    import torch
    src = np.zeros(len(pos), dtype=np.dtype(L.Src))
    p = np.asarray(pos, np.float64)
    src["x"], src["y"], src["z"] = p[:, 0], p[:, 1], p[:, 2]
    src["m"] = np.asarray(mass, np.float32)
    return torch.from_numpy(src.view(np.uint8).reshape(-1).copy()).to(device)


def direct_sum(pos, mass, eps, targets, device="cuda"):
    """FP64 direct sum on the device (otoo_direct) for the given particle
    indices (caller order): returns (acc [k][3], pot [k]) as numpy."""
    import torch
    src = _particle_sources(pos, mass, device)
    t = torch.from_numpy(np.ascontiguousarray(targets, np.int64)).to(device)
    n, nt = len(pos), int(t.shape[0])
    nch = int(L.load().otoo_direct_chunks(n, nt))
    scratch = torch.empty(4 * nch * nt, dtype=torch.float64, device=device)
    acc = torch.empty((nt, 3), dtype=torch.float64, device=device)
    pot = torch.empty(nt, dtype=torch.float64, device=device)
    status = torch.zeros(1, dtype=torch.int32, device=device)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.call("otoo_direct", src.data_ptr(), n, t.data_ptr(), nt, float(eps) ** 2, acc.data_ptr(), pot.data_ptr(),
           scratch.data_ptr(), status.data_ptr(), st)
    torch.cuda.synchronize()
    assert int(status.item()) == 0, "otoo_direct: target index out of range"
    return acc.cpu().numpy(), pot.cpu().numpy()


def sph_direct(pos, mass, h, targets, device="cuda"):
    """FP64 brute-force SPH density on the device (otoo_sph_direct) for the
    given particle indices (caller order)."""
    import torch
    src = _particle_sources(pos, mass, device)
    hd = torch.from_numpy(np.ascontiguousarray(h, np.float32)).to(device)
    t = torch.from_numpy(np.ascontiguousarray(targets, np.int64)).to(device)
    rho = torch.empty(int(t.shape[0]), dtype=torch.float64, device=device)
    status = torch.zeros(1, dtype=torch.int32, device=device)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.call("otoo_sph_direct", src.data_ptr(), hd.data_ptr(), len(pos), t.data_ptr(), int(t.shape[0]),
           rho.data_ptr(), status.data_ptr(), st)
    torch.cuda.synchronize()
    assert int(status.item()) == 0, "otoo_sph_direct: target index out of range"
    return rho.cpu().numpy()


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


def _stream(stream, device):
    import torch
    st = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(st.cuda_stream)


class BufferPool:
    """Device buffers kept between steps (grown when too small), so that a
    loop of device walks and force steps reuses the same memory and the
    force step's recorded graph."""

    def __init__(self, device):
        self.device = device
        self.bufs = {}
        self.meta = {}

    def get(self, name, n, dtype):
        import torch
        t = self.bufs.get(name)
        if t is None or t.dtype != dtype or t.numel() < n:
            t = torch.empty(max(int(n), 1), dtype=dtype, device=self.device)
            self.bufs[name] = t
        return t[:max(int(n), 1)]


def _alloc(pool, device):
    import torch
    if pool is None:
        return lambda name, n, dtype: torch.empty(max(int(n), 1), dtype=dtype, device=device)
    return pool.get


class DeviceTree:
    """Inputs of the device walk for one tree, uploaded once: sources and
    quadrupoles (as the host lists store them), walk records
    (otoo_tree_device_arrays), the group ranges (otoo_find_groups) and the
    tree-to-caller permutation."""

    def __init__(self, tree, n_crit, use_quad=True, device="cuda", mac="theta", delta=0.0, m_limit=0.0, h_sph=None):
        v = L.TreeView()
        L.call("otoo_tree_export", tree._h, ctypes.byref(v))
        n, nc = int(v.n_part), int(v.n_cell)
        src = np.empty(n + nc, np.dtype(L.Src))
        quad = np.empty(nc, np.dtype(L.Quad))
        cell = np.empty(nc, np.dtype(L.WCell))
        cell64 = np.empty(nc, np.dtype(L.WCell64))
        hs = None if h_sph is None else np.ascontiguousarray(h_sph, dtype=np.float32)
        p = _params(0.0, tree.leaf_size, n_crit, use_quad, 1.0, None, mac, delta, m_limit, hs)
        L.call("otoo_tree_device_arrays", tree._h, int(bool(use_quad)), ctypes.byref(p), src.ctypes.data,
               quad.ctypes.data, cell.ctypes.data, cell64.ctypes.data)
        self.mac = p.mac
        G = ctypes.c_int64()
        L.call("otoo_find_groups", tree._h, int(n_crit), None, None, 0, ctypes.byref(G))
        first = np.empty(G.value, np.int32)
        count = np.empty(G.value, np.int32)
        L.call("otoo_find_groups", tree._h, int(n_crit), first.ctypes.data, count.ctypes.data, G.value,
               ctypes.byref(G))
        self.n_part, self.n_cell, self.n_groups = n, nc, int(G.value)
        self.n_src = n + nc
        self.use_quad = bool(use_quad)
        self.n_crit = int(n_crit)
        self.device = device
        perm = L.view(v.perm, np.int64, (n,))
        self.bufs = dict(src=_to_dev(src, device), quad=_to_dev(quad, device) if use_quad else None,
                         cell=_to_dev(cell, device), cell64=_to_dev(cell64, device),
                         first=_to_dev(first, device), count=_to_dev(count, device), perm=_to_dev(perm, device))
        self._tree = tree

    @classmethod
    def build(cls, pos, mass, leaf_size, n_crit, use_quad=True, device="cuda", mac="theta", delta=0.0, m_limit=0.0,
              cap_cell=None, stream=None, h_sph=None):
        """The tree built on the device (otoo_devtree_build) from positions
        [n][3] FP64 and masses [n] FP32 (numpy arrays or device tensors,
        caller order); the cell capacity grows until the tree fits."""
        import torch
        self = cls.__new__(cls)
        if torch.is_tensor(pos):
            pos_d = pos.to(device=device, dtype=torch.float64).contiguous()
        else:
            pos_d = torch.from_numpy(np.ascontiguousarray(pos, dtype=np.float64)).to(device)
        if torch.is_tensor(mass):
            mass_d = mass.to(device=device, dtype=torch.float32).contiguous()
        else:
            mass_d = torch.from_numpy(np.ascontiguousarray(mass, dtype=np.float32)).to(device)
        n = int(pos_d.shape[0])
        h_d = None
        if h_sph is not None:
            h_d = (h_sph.to(device=device, dtype=torch.float32).contiguous() if torch.is_tensor(h_sph)
                   else torch.from_numpy(np.ascontiguousarray(h_sph, dtype=np.float32)).to(device))
        cap = int(cap_cell) if cap_cell else max(1024, n)
        st = _stream(stream, device)
        u8, i32, i64 = torch.uint8, torch.int32, torch.int64
        while True:
            b = dict(src=torch.empty((n + cap) * 32, dtype=u8, device=device),
                     quad=torch.empty(cap * 32, dtype=u8, device=device),
                     cell=torch.empty(cap * 64, dtype=u8, device=device),
                     cell64=torch.empty(cap * 96, dtype=u8, device=device),
                     first=torch.empty(n, dtype=i32, device=device), count=torch.empty(n, dtype=i32, device=device),
                     perm=torch.empty(n, dtype=i64, device=device), level=torch.empty(cap, dtype=i32, device=device),
                     status=torch.zeros(2, dtype=i32, device=device))
            t = L.DevTree()
            t.n_part, t.cap_cell, t.leaf_size, t.n_crit = n, cap, int(leaf_size), int(n_crit)
            t.use_quad, t.mac = int(bool(use_quad)), MAC_KINDS[mac]
            t.delta, t.m_limit = float(delta), float(m_limit)
            t.h_sph = h_d.data_ptr() if h_d is not None else None
            t.src, t.quad, t.cell, t.cell64 = (b[k].data_ptr() for k in ("src", "quad", "cell", "cell64"))
            t.group_first, t.group_count, t.perm = b["first"].data_ptr(), b["count"].data_ptr(), b["perm"].data_ptr()
            t.cell_level, t.status = b["level"].data_ptr(), b["status"].data_ptr()
            nbytes = int(L.load().otoo_devtree_scratch_bytes(n, cap))
            scratch = torch.empty(nbytes, dtype=u8, device=device)
            try:
                L.call("otoo_devtree_build", pos_d.data_ptr(), mass_d.data_ptr(), ctypes.byref(t), scratch.data_ptr(),
                       nbytes, st)
                break
            except L.OtooError as e:
                if e.code != L.OTOO_ENOMEM:
                    raise
                cap *= 2
        del scratch
        nc, G = int(t.n_cell), int(t.n_groups)
        self.n_part, self.n_cell, self.n_groups = n, nc, G
        self.n_src = n + nc
        self.use_quad = bool(use_quad)
        self.n_crit = int(n_crit)
        self.device = device
        self.mac = t.mac
        self.depth = int(t.depth)
        self.root_lo, self.root_side = np.array(t.root_lo), float(t.root_side)
        self.bufs = dict(src=b["src"][:(n + nc) * 32], quad=b["quad"][:nc * 32] if use_quad else None,
                         cell=b["cell"][:nc * 64], cell64=b["cell64"][:nc * 96], first=b["first"][:G],
                         count=b["count"][:G], perm=b["perm"], level=b["level"][:nc])
        self._tree = None
        return self

    def h2d_bytes(self):
        return sum(b.numel() for b in self.bufs.values() if b is not None)

    def fused(self, theta, eps, iblock=2, theta_per_group=None, pool=None):
        """The walk fused with the FP32 force (FusedStep); every group at most
        32 * iblock particles."""
        return FusedStep(self, theta, eps, iblock, theta_per_group, pool)

    def walk(self, theta, eps, theta_per_group=None, exact=False, stream=None, pool=None, max_entries=None,
             single=True, group_set=0):
        """Groups and lists on the device.  Without a BufferPool: two passes
        (otoo_walk_count, otoo_walk_fill) into a dense list.  With one, the
        buffers of the previous walk are reused (and overwritten), and once a
        walk has set the slot sizes (1.25 x its largest n_cell / n_part) the
        walk is one pass (otoo_walk_single) whose slots serve as the list,
        falling back to two passes when a group outgrows its slot.
        max_entries: raise ValueError instead of allocating a longer list.
        group_set: groups one warp walks together (1..8; 0 = as many as
        keep every resident warp busy, up to 8); same entries per group."""
        return DeviceLists(self, theta, eps, theta_per_group, exact, stream, pool, max_entries, single, group_set)


class FusedStep:
    """The walk fused with the FP32 force (otoo_walk_force): one warp per
    group walks the tree and evaluates each tile of its entries as it is
    found; no list, no plan.  Outputs in caller order."""

    def __init__(self, dtree, theta, eps, iblock=2, theta_per_group=None, pool=None):
        import torch
        dev = dtree.device
        G = dtree.n_groups
        alloc = _alloc(pool, dev)
        self.tree = dtree
        self.iblock = int(iblock)
        b = dict(counter=alloc("fcounter", 4, torch.int32),
                 totals=alloc("ftotals", L.load().otoo_walk_totals_len(G), torch.int64),
                 split=alloc("fsplit", 8 * dtree.n_src, torch.float32))
        if theta_per_group is not None:
            tpg = np.ascontiguousarray(theta_per_group, dtype=np.float32)
            assert tpg.shape == (G,)
            b["tpg"] = alloc("ftpg", G, torch.float32)
            b["tpg"].copy_(torch.from_numpy(tpg))
        w = L.DevWalk()
        w.n_part, w.n_cell, w.n_groups, w.exact = dtree.n_part, dtree.n_cell, G, 0
        w.mac = dtree.mac
        w.theta, w.eps2 = float(theta), float(eps) * float(eps)
        tb = dtree.bufs
        w.src, w.cell, w.cell64 = tb["src"].data_ptr(), tb["cell"].data_ptr(), tb["cell64"].data_ptr()
        w.group_first, w.group_count = tb["first"].data_ptr(), tb["count"].data_ptr()
        w.theta_per_group = b["tpg"].data_ptr() if "tpg" in b else None
        w.counter, w.totals = b["counter"].data_ptr(), b["totals"].data_ptr()
        self.struct = w
        self.bufs = b

    def __call__(self, accel, pot, stream=None, check=True):
        """Enqueues one step into accel [n][3] and pot [n] (FP64 device
        tensors); with check, waits and raises on a device-side error."""
        st = _stream(stream, self.tree.device)
        tb = self.tree.bufs
        quad = tb["quad"].data_ptr() if tb.get("quad") is not None else None
        L.call("otoo_walk_force", ctypes.byref(self.struct), quad, tb["perm"].data_ptr(),
               self.bufs["split"].data_ptr(), self.iblock, accel.data_ptr(), pot.data_ptr(), st)
        if check:
            L.call("otoo_walk_check_status", ctypes.byref(self.struct), st)

    def totals(self):
        """(list entries, interactions, cell interactions) of the last step."""
        t = [int(x) for x in self.bufs["totals"][:3].tolist()]
        return tuple(t)


class DeviceLists:
    """Groups and lists made by the device walk (device buffers).  bufs["list"]
    holds list_len entries: the dense list of the two-pass walk (list_len =
    n_list), or the slots of the one-pass walk (in_place; each group's
    entries contiguous inside its slot, cells in reverse walk order)."""

    SLOT_BYTES_MAX = 24 << 30  # device memory the one-pass walk's slots may take

    def __init__(self, dtree, theta, eps, theta_per_group=None, exact=False, stream=None, pool=None,
                 max_entries=None, single=True, group_set=0):
        import torch
        dev = dtree.device
        G = dtree.n_groups
        self.tree = dtree
        self.pool = pool
        self.n_part, self.n_src, self.n_groups = dtree.n_part, dtree.n_src, G
        self.use_quad = dtree.use_quad
        alloc = _alloc(pool, dev)
        b = dict(groups=alloc("groups", G * 64, torch.uint8), counter=alloc("wcounter", 4, torch.int32),
                 totals=alloc("totals", L.load().otoo_walk_totals_len(G), torch.int64))
        if theta_per_group is not None:
            tpg = np.ascontiguousarray(theta_per_group, dtype=np.float32)
            assert tpg.shape == (G,)
            b["tpg"] = alloc("tpg", G, torch.float32)
            b["tpg"].copy_(torch.from_numpy(tpg))
        w = L.DevWalk()
        w.n_part, w.n_cell, w.n_groups, w.exact = dtree.n_part, dtree.n_cell, G, int(bool(exact))
        w.mac = dtree.mac
        w.set = int(group_set)
        w.theta, w.eps2 = float(theta), float(eps) * float(eps)
        tb = dtree.bufs
        w.src, w.cell, w.cell64 = tb["src"].data_ptr(), tb["cell"].data_ptr(), tb["cell64"].data_ptr()
        w.group_first, w.group_count = tb["first"].data_ptr(), tb["count"].data_ptr()
        w.theta_per_group = b["tpg"].data_ptr() if "tpg" in b else None
        w.counter, w.totals = b["counter"].data_ptr(), b["totals"].data_ptr()
        self.struct = w
        self.bufs = b
        st = _stream(stream, dev)
        gp = b["groups"].data_ptr()
        key = (dtree.n_groups, dtree.mac)
        slots = pool.meta.get(key) if (pool is not None and single) else None
        self.slots = None
        if slots:
            ccap, pcap = slots
            spool = alloc("slots", G * (ccap + pcap), torch.int32)
            L.call("otoo_walk_single", ctypes.byref(w), gp, spool.data_ptr(), ccap, pcap, st)
        tot = [int(x) for x in b["totals"][:6].tolist()] if slots else None
        self.one_pass = bool(slots) and tot[5] == 0
        if not self.one_pass:
            L.call("otoo_walk_count", ctypes.byref(w), gp, st)
            tot = [int(x) for x in b["totals"][:6].tolist()]
        self.n_list, self.interactions, self.cell_interactions = tot[:3]
        if max_entries is not None and self.n_list > max_entries:
            raise ValueError("walk: %d list entries exceed max_entries %d" % (self.n_list, max_entries))
        if self.one_pass:
            self.slots = (ccap, pcap)
            b["list"] = spool
            self.list_len = G * (ccap + pcap)
        else:
            b["list"] = alloc("list", self.n_list, torch.int32)
            self.list_len = self.n_list
            L.call("otoo_walk_fill", ctypes.byref(w), gp, b["list"].data_ptr(), self.n_list, st)
        L.call("otoo_walk_check_status", ctypes.byref(w), st)
        if pool is not None and single:
            ccap, pcap = int(1.25 * tot[3]) + 64, int(1.25 * tot[4]) + 64
            if 4 * G * (ccap + pcap) <= self.SLOT_BYTES_MAX:
                pool.meta[key] = (ccap, pcap)

    @property
    def groups(self):
        """Group records copied to the host (numpy structured array)."""
        return self.bufs["groups"].cpu().numpy().view(np.dtype(L.Group))

    @property
    def in_place(self):
        return self.slots is not None

    @property
    def list(self):
        """The dense list on the host, in group order with each group's cells
        in walk order (what otoo_walk_fill writes), whichever layout the
        device holds."""
        if not self.in_place:
            return self.bufs["list"][:self.n_list].cpu().numpy()
        g = self.groups
        raw = self.bufs["list"].cpu().numpy()
        nc = g["n_cell"].astype(np.int64)
        ln = nc + g["n_part"]
        gi = np.repeat(np.arange(len(g)), ln)
        k = np.arange(int(ln.sum()), dtype=np.int64) - np.repeat(np.cumsum(ln) - ln, ln)
        src = g["list_off"][gi] + np.where(k < nc[gi], nc[gi] - 1 - k, k)
        return raw[src]

    def compact(self, stream=None):
        """Moves the lists of a one-pass walk into a dense device list in
        group order (otoo_walk_compact: the list and offsets the two-pass walk
        writes); nothing to do for a dense list."""
        import torch
        if not self.in_place:
            return self
        st = _stream(stream, self.tree.device)
        ccap, pcap = self.slots
        dense = _alloc(self.pool, self.tree.device)("list", self.n_list, torch.int32)
        L.call("otoo_walk_compact", ctypes.byref(self.struct), self.bufs["groups"].data_ptr(),
               self.bufs["list"].data_ptr(), ccap, pcap, dense.data_ptr(), self.n_list, st)
        L.call("otoo_walk_check_status", ctypes.byref(self.struct), st)
        self.bufs["list"], self.list_len, self.slots = dense, self.n_list, None
        return self

    def plan(self, tune, stream=None):
        return DevicePlan(self, tune, stream)


class DevicePlan:
    """Work items made on the device (otoo_plan_count + otoo_plan_fill)."""

    def __init__(self, dl, tune, stream=None):
        import torch
        dev = dl.tree.device
        G = dl.n_groups
        self.tune = tune
        st = _stream(stream, dev)
        alloc = _alloc(dl.pool, dev)
        scratch = alloc("pscratch", L.load().otoo_plan_scratch_ints(G), torch.int32)
        ptot = alloc("ptotals", 4, torch.int64)
        gp = dl.bufs["groups"].data_ptr()
        L.call("otoo_plan_count", gp, G, ctypes.byref(tune), scratch.data_ptr(), ptot.data_ptr(), st)
        n_items, n_splits, slots, ncm = (int(x) for x in ptot.tolist())
        self.n_items, self.n_splits, self.n_crit_max = n_items, n_splits, max(ncm, 1)
        self.partial_doubles = slots * 4 * self.n_crit_max
        self.items_buf = alloc("items", n_items * 32, torch.uint8)
        self.splits_buf = alloc("splits", n_splits * 16, torch.uint8)
        L.call("otoo_plan_fill", gp, G, ctypes.byref(tune), scratch.data_ptr(), ptot.data_ptr(),
               self.items_buf.data_ptr(), n_items, self.splits_buf.data_ptr(), n_splits,
               dl.bufs["counter"].data_ptr(), st)
        L.call("otoo_walk_check_status", ctypes.byref(dl.struct), st)

    @property
    def items(self):
        return self.items_buf[:self.n_items * 32].cpu().numpy().view(np.dtype(L.Item))

    @property
    def splits(self):
        return self.splits_buf[:self.n_splits * 16].cpu().numpy().view(np.dtype(L.Split))


class DeviceStep:
    """A force step whose lists and plan were made on the device; usable
    with force() like a DeviceSystem."""

    def __init__(self, dl, plan, use_perm=True):
        import torch
        dev = dl.tree.device
        tb = dl.tree.bufs
        alloc = _alloc(dl.pool, dev)
        self.lists, self.plan = dl, plan
        self.bufs = dict(src=tb["src"], quad=tb["quad"], groups=dl.bufs["groups"], list=dl.bufs["list"],
                         items=plan.items_buf, splits=plan.splits_buf if plan.n_splits else None,
                         perm=tb["perm"] if use_perm else None,
                         partial=alloc("partial", plan.partial_doubles, torch.float64),
                         counter=alloc("fcounter", 4, torch.int32),
                         split=alloc("split", dl.n_src * 8, torch.float32))
        s = L.DevSystem()
        s.n_part, s.n_src, s.n_list = dl.n_part, dl.n_src, dl.list_len
        s.partial_doubles = self.bufs["partial"].numel()
        s.n_groups, s.n_items, s.n_splits, s.n_crit_max = dl.n_groups, plan.n_items, plan.n_splits, plan.n_crit_max
        for k in ("src", "quad", "groups", "list", "items", "splits", "perm", "partial", "counter", "split"):
            setattr(s, k, self.bufs[k].data_ptr() if self.bufs[k] is not None else None)
        self.struct = s

    @property
    def n_part(self):
        return self.lists.n_part

    @property
    def tune(self):
        return self.plan.tune
