"""ctypes binding of libotoo.so: the C ABI of include/otoo.h with the same
names, argument marshalling only.  Loading fails loudly when the library is
missing; there is no fallback implementation."""
from __future__ import annotations

import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libotoo.so")

OTOO_OK = 0
OTOO_EINVAL = -1
OTOO_ENOMEM = -2
OTOO_ECUDA = -3
OTOO_EDEVICE = -4
OTOO_FP32K = 0
OTOO_FP64 = 1
MLP_IN = 6
MLP_H = 32
MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_H + 1

i32, i64, f32, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
vp = ctypes.c_void_p


class OtooError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("otoo error %d: %s" % (code, msg))
        self.code = code


OTOO_MAC_THETA = 0
OTOO_MAC_SW = 1
OTOO_MAC_SPH = 2


class Params(ctypes.Structure):
    _fields_ = [("theta", f64), ("leaf_size", i32), ("n_crit", i32), ("use_quad", i32), ("mac", i32),
                ("eps", f64), ("theta_per_group", ctypes.POINTER(f32)), ("delta", f64), ("m_limit", f64),
                ("h_sph", vp)]


class Tune(ctypes.Structure):
    _fields_ = [("block", i32), ("iblock", i32), ("tile", i32), ("split", i32), ("ctas_per_sm", i32),
                ("packed", i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Src(ctypes.Structure):
    _fields_ = [("x", f64), ("y", f64), ("z", f64), ("m", f32), ("pad", i32)]


class Quad(ctypes.Structure):
    _fields_ = [(k, f32) for k in ("xx", "yy", "zz", "xy", "xz", "yz", "b2", "pad")]


class Group(ctypes.Structure):
    _fields_ = [("first", i32), ("count", i32), ("n_cell", i32), ("n_part", i32), ("list_off", i64),
                ("eps2", f64), ("cx", f64), ("cy", f64), ("cz", f64), ("theta", f32), ("sys", i32)]


class Item(ctypes.Structure):
    _fields_ = [("g", i32), ("i0", i32), ("ni", i32), ("j0", i32), ("j1", i32), ("slot", i32), ("pad0", i32),
                ("pad1", i32)]


class Split(ctypes.Structure):
    _fields_ = [("g", i32), ("slot0", i32), ("n_chunks", i32), ("pad", i32)]


class DevSystem(ctypes.Structure):
    _fields_ = [("n_part", i64), ("n_src", i64), ("n_list", i64), ("partial_doubles", i64), ("n_groups", i32),
                ("n_items", i32), ("n_splits", i32), ("n_crit_max", i32), ("src", vp), ("quad", vp), ("groups", vp),
                ("list", vp), ("items", vp), ("splits", vp), ("perm", vp), ("partial", vp), ("counter", vp),
                ("split", vp)]


class ListsView(ctypes.Structure):
    _fields_ = [("n_part", i64), ("n_src", i64), ("n_groups", i64), ("n_list", i64), ("n_sys", i32),
                ("use_quad", i32), ("src", vp), ("quad", vp), ("groups", vp), ("list", vp), ("perm", vp),
                ("sys_part_off", vp), ("interactions", i64), ("cell_interactions", i64)]


class PlanInfo(ctypes.Structure):
    _fields_ = [("n_items", i64), ("n_splits", i64), ("partial_doubles", i64), ("n_crit_max", i32),
                ("pad", i32), ("items", vp), ("splits", vp)]


class TreeView(ctypes.Structure):
    _fields_ = [("n_part", i64), ("n_cell", i64), ("depth", i32), ("leaf_size", i32),
                ("root_lo", f64 * 3), ("root_side", f64), ("pos", vp), ("mass", vp), ("perm", vp),
                ("cell_begin", vp), ("cell_end", vp), ("cell_level", vp), ("cell_nchild", vp),
                ("cell_child0", vp), ("cell_org", vp), ("cell_com", vp), ("cell_mass", vp), ("cell_quad", vp),
                ("cell_b2", vp), ("cell_bmax", vp)]


class WCell(ctypes.Structure):
    _fields_ = [("com_hi", f32 * 3), ("com_lo", f32 * 3), ("e", f32 * 3), ("side", f32), ("s", f32),
                ("child0", i32), ("nchild", i32), ("begin", i32), ("end", i32), ("rb", f32)]


class WCell64(ctypes.Structure):
    _fields_ = [("lo", f64 * 3), ("side", f64), ("com", f64 * 3), ("gc", f64 * 3), ("rb", f64), ("pad", f64)]


class DevWalk(ctypes.Structure):
    _fields_ = [("n_part", i64), ("n_cell", i64), ("n_groups", i32), ("exact", i32), ("mac", i32), ("set", i32),
                ("theta", f64),
                ("eps2", f64), ("src", vp), ("cell", vp), ("cell64", vp), ("group_first", vp),
                ("group_count", vp), ("theta_per_group", vp), ("counter", vp), ("totals", vp)]


class ThetaNet(ctypes.Structure):
    _fields_ = [("wbf16", vp), ("mean", vp), ("std", vp), ("lo", vp), ("hi", vp)]


class ThetaRule(ctypes.Structure):
    _fields_ = [("theta0", f32), ("target_rms", f32), ("calib", f32), ("alpha", f32), ("beta", f32),
                ("fallback", f32)]


class DevTree(ctypes.Structure):
    _fields_ = [("n_part", i64), ("cap_cell", i64), ("leaf_size", i32), ("n_crit", i32), ("use_quad", i32),
                ("mac", i32), ("delta", f64), ("m_limit", f64), ("h_sph", vp), ("n_cell", i64), ("n_groups", i64), ("depth", i32),
                ("pad", i32), ("root_lo", f64 * 3), ("root_side", f64), ("src", vp), ("quad", vp), ("cell", vp),
                ("cell64", vp), ("group_first", vp), ("group_count", vp), ("perm", vp), ("cell_level", vp),
                ("status", vp)]


for _s, _n in ((Src, 32), (Quad, 32), (Group, 64), (Item, 32), (Split, 16), (WCell, 64), (WCell64, 96)):
    assert ctypes.sizeof(_s) == _n, (_s, ctypes.sizeof(_s))

# name -> (argtypes); every function returns int unless listed in _VOID
_SIGS = {
    "otoo_build_tree": [vp, vp, i64, ctypes.POINTER(Params), ctypes.POINTER(vp)],
    "otoo_make_groups_and_lists": [vp, ctypes.POINTER(Params), ctypes.POINTER(vp)],
    "otoo_pack_batch": [ctypes.POINTER(vp), i32, ctypes.POINTER(vp)],
    "otoo_make_plan": [vp, ctypes.POINTER(Tune), ctypes.POINTER(vp)],
    "otoo_lists_export": [vp, ctypes.POINTER(ListsView)],
    "otoo_plan_export": [vp, ctypes.POINTER(PlanInfo)],
    "otoo_tree_export": [vp, ctypes.POINTER(TreeView)],
    "otoo_group_features": [vp, vp, vp],
    "otoo_tree_free": [vp],
    "otoo_lists_free": [vp],
    "otoo_plan_free": [vp],
    "otoo_default_tune": [i32, ctypes.POINTER(Tune)],
    "otoo_force": [ctypes.POINTER(DevSystem), vp, vp, i32, ctypes.POINTER(Tune), vp],
    "otoo_force_host": [ctypes.POINTER(ListsView), ctypes.POINTER(PlanInfo), vp, vp, i32, ctypes.POINTER(Tune), vp],
    "otoo_check_status": [ctypes.POINTER(DevSystem), vp],
    "otoo_centre_relative": [vp, i64, ctypes.POINTER(f64), vp, vp, vp],
    "otoo_force_static": [ctypes.POINTER(DevSystem), i64, vp, vp, i32, ctypes.POINTER(Tune), vp],
    "otoo_force_static_capacity": [],
    "otoo_force_static_status": [vp],
    "otoo_fma_probe_threads": [],
    "otoo_fma_probe": [i32, i32, vp, ctypes.POINTER(f64), vp],
    "otoo_direct_chunks": [i64, i64],
    "otoo_direct": [vp, i64, vp, i64, f64, vp, vp, vp, vp, vp],
    "otoo_mlp_predict": [vp, vp, vp, i64, vp],
    "otoo_mlp_scratch_floats": [i64],
    "otoo_mlp_grad": [vp, vp, vp, i64, vp, vp, vp, vp],
    "otoo_mlp_train_step": [vp, vp, vp, vp, vp, vp, vp, i64, f32, f32, f32, f32, i32, vp, vp],
    "otoo_mlp_to_bf16": [vp, vp, i32, vp],
    "otoo_select_theta": [vp, vp, vp, i32, i64, f32, vp, f32, vp, vp],
    "otoo_learned_theta_scratch_floats": [i64],
    "otoo_mlp_standardise": [vp, i64, vp, vp, vp, vp],
    "otoo_learned_theta": [ctypes.POINTER(ThetaNet), ctypes.POINTER(ThetaRule), vp, vp, i64, vp, i32, vp, vp, vp, vp],
    "otoo_group_rms_error": [vp, vp, vp, i64, f32, vp, vp, vp],
    "otoo_find_groups": [vp, i32, vp, vp, i64, ctypes.POINTER(i64)],
    "otoo_tree_device_arrays": [vp, i32, ctypes.POINTER(Params), vp, vp, vp, vp],
    "otoo_walk_totals_len": [i64],
    "otoo_walk_count": [ctypes.POINTER(DevWalk), vp, vp],
    "otoo_walk_fill": [ctypes.POINTER(DevWalk), vp, vp, i64, vp],
    "otoo_walk_check_status": [ctypes.POINTER(DevWalk), vp],
    "otoo_walk_force": [ctypes.POINTER(DevWalk), vp, vp, vp, i32, vp, vp, vp],
    "otoo_walk_single": [ctypes.POINTER(DevWalk), vp, vp, i64, i64, vp],
    "otoo_walk_compact": [ctypes.POINTER(DevWalk), vp, vp, i64, i64, vp, i64, vp],
    "otoo_plan_scratch_ints": [i64],
    "otoo_plan_count": [vp, i32, ctypes.POINTER(Tune), vp, vp, vp],
    "otoo_plan_fill": [vp, i32, ctypes.POINTER(Tune), vp, vp, vp, i64, vp, i64, vp, vp],
    "otoo_sph_density": [ctypes.POINTER(DevSystem), vp, vp, ctypes.POINTER(Tune), vp],
    "otoo_sph_direct": [vp, vp, i64, vp, i64, vp, vp, vp],
    "otoo_devtree_scratch_bytes": [i64, i64],
    "otoo_devtree_build": [vp, vp, ctypes.POINTER(DevTree), vp, i64, vp],
    "otoo_last_error": [],
}
_RET_I64 = {"otoo_mlp_scratch_floats", "otoo_learned_theta_scratch_floats", "otoo_force_static_capacity", "otoo_fma_probe_threads", "otoo_direct_chunks", "otoo_walk_totals_len",
            "otoo_plan_scratch_ints", "otoo_devtree_scratch_bytes"}
_VOID = {"otoo_tree_free", "otoo_lists_free", "otoo_plan_free"}
_OPTIONAL = set()

_lib = None


def load():
    """Load libotoo.so (built by __graft_entry__.build() / build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libotoo.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, args in _SIGS.items():
        if not hasattr(lib, name):
            if name in _OPTIONAL:
                continue
            raise ImportError("libotoo.so lacks %s" % name)
        fn = getattr(lib, name)
        fn.argtypes = args
        if name in _VOID:
            fn.restype = None
        elif name == "otoo_last_error":
            fn.restype = ctypes.c_char_p
        elif name in _RET_I64:
            fn.restype = i64
        else:
            fn.restype = ctypes.c_int
    _lib = lib
    return lib


def check(rc):
    if rc != OTOO_OK:
        raise OtooError(rc, load().otoo_last_error().decode())
    return rc


def call(name, *args):
    return check(getattr(load(), name)(*args))


def ptr(a):
    """Address of a numpy array or torch tensor (data pointer)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def view(addr, dtype, shape):
    """numpy view (no copy) of library-owned host memory."""
    n = int(np.prod(shape))
    if n == 0:
        return np.zeros(shape, dtype)
    buf = (ctypes.c_char * (n * np.dtype(dtype).itemsize)).from_address(addr)
    return np.frombuffer(buf, dtype=dtype, count=n).reshape(shape)


def structs_dtype(st):
    """numpy structured dtype matching a ctypes Structure."""
    return np.dtype(st)


def default_tune(n_crit):
    t = Tune()
    call("otoo_default_tune", n_crit, ctypes.byref(t))
    return t
