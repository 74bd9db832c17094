"""The two precision devices the FP32 force form rests on, checked on the GPU
through the C ABI against FP64 arithmetic done here:

* the centre-relative conversion: each coordinate is split once per step
  into a float pair (hi, lo) and staged as (hi - c) + lo in FP32, c the group
  centre rounded to FP32 (otoo_centre_relative runs the force kernels' own
  split and staging function);
* the compensated accumulation: per-tile FP32 sums added into Kahan sums,
  which keeps the many small terms a plain FP32 running sum drops once a
  large term has been added.

Bounds: u(v) is the spacing of FP32 numbers at |v|.  A near entry (hi within
a factor of two of c, so hi - c is exact) is the FP64 difference x - c
rounded once, up to the rounding of lo: |got - ref| <= u(ref)/2 + 2^-47 |x|.
Any entry: |got - ref| <= 2 u(ref) + 2^-47 |x| (two roundings).  A plain FP32
conversion, fl(fl(x) - c), errs by up to u(x)/2, far above both for entries
close to c."""
import ctypes

import numpy as np
import pytest

from paper_1206_1199_gb300 import _lib as L
from paper_1206_1199_gb300 import ic, system as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as t
    L.load()
    return t


def ulp32(v):
    return np.spacing(np.abs(np.asarray(v, np.float64)).astype(np.float32)).astype(np.float64)


def centre_relative(torch, pos, c):
    n = len(pos)
    src = np.zeros(n, np.dtype(L.Src))
    src["x"], src["y"], src["z"] = pos[:, 0], pos[:, 1], pos[:, 2]
    src["m"] = 1.0
    d_src = torch.from_numpy(src.view(np.uint8).copy()).cuda()
    out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    scratch = torch.empty(8 * n, dtype=torch.float32, device="cuda")
    cc = (ctypes.c_double * 3)(*c)
    L.call("otoo_centre_relative", d_src.data_ptr(), n, cc, out.data_ptr(), scratch.data_ptr(),
           ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("c", [(1234.567890123456, -0.0123456789, 3.0e5), (0.75, -7.5, 1.0e-3),
                               (-8.0e6, 2.0 ** 20, -1.0), (0.0, 0.0, 0.0)])
def test_centre_relative_conversion_is_the_fp64_difference_rounded(torch, c):
    rng = np.random.default_rng(31)
    c = np.array(c)
    c32 = c.astype(np.float32).astype(np.float64)
    n = 60000
    # near entries: offsets from 1e-12 to 0.4 of |c| (within a factor of two
    # of c), both signs, plus entries exactly representable in FP32
    rel = np.exp(rng.uniform(np.log(1e-12), np.log(0.4), (n, 3))) * rng.choice([-1.0, 1.0], (n, 3))
    scale = np.maximum(np.abs(c32), 1e-30)
    near = c32 + rel * scale
    near[:1000] = near[:1000].astype(np.float32).astype(np.float64)
    # far entries: anywhere within 10^4 |c| (and around 0)
    far = rng.uniform(-1.0, 1.0, (n, 3)) * 10.0 ** rng.uniform(-6, 4, (n, 1)) * np.maximum(np.abs(c32), 1.0)
    cases = ((far, False),) if np.any(c32 == 0) else ((near, True), (far, False))
    for pos, near_bound in cases:
        got = centre_relative(torch, pos, c)
        ref = pos - c32                     # exact in FP64 for near entries
        err = np.abs(got - ref)
        slack = 2.0 ** -47 * np.abs(pos)
        hi = pos.astype(np.float32).astype(np.float64)
        sterbenz = (hi * c32 > 0) & (np.abs(hi) <= 2 * np.abs(c32)) & (np.abs(c32) <= 2 * np.abs(hi))
        if near_bound:
            assert sterbenz.mean() > 0.99
            m = sterbenz
            assert np.all(err[m] <= 0.5 * ulp32(ref[m]) * (1 + 2.0 ** -20) + slack[m])
            # representable coordinates (lo = 0): exactly fl32(x - c)
            exact = (hi == pos) & m
            assert exact.sum() > 2000
            np.testing.assert_array_equal(got[exact], ref[exact].astype(np.float32).astype(np.float64))
            # a plain FP32 conversion would not meet the bound
            plain = (pos.astype(np.float32) - c32.astype(np.float32)).astype(np.float64)
            assert np.mean(np.abs(plain - ref) > 0.5 * ulp32(ref) + slack) > 0.5
        assert np.all(err <= 2.0 * ulp32(ref) + slack), np.max(err / (ulp32(ref) + slack))


def hand_system(torch, pos, mass, list_idx, ni, eps, centre):
    """Device inputs of one group of ni targets (sources 0..ni-1) with the
    given list (particle entries only) and one work item over all of it."""
    n = len(pos)
    src = np.zeros(n, np.dtype(L.Src))
    src["x"], src["y"], src["z"] = pos[:, 0], pos[:, 1], pos[:, 2]
    src["m"] = mass
    grp = np.zeros(1, np.dtype(L.Group))
    grp["first"], grp["count"], grp["n_cell"], grp["n_part"] = 0, ni, 0, len(list_idx)
    grp["list_off"], grp["eps2"] = 0, eps * eps
    grp["cx"], grp["cy"], grp["cz"] = centre
    grp["theta"] = 0.0
    item = np.zeros(1, np.dtype(L.Item))
    item["g"], item["i0"], item["ni"], item["j0"], item["j1"], item["slot"] = 0, 0, ni, 0, len(list_idx), -1
    b = {k: torch.from_numpy(np.ascontiguousarray(v).view(np.uint8).copy()).cuda()
         for k, v in (("src", src), ("groups", grp), ("list", np.asarray(list_idx, np.int32)), ("items", item))}
    b["counter"] = torch.zeros(4, dtype=torch.int32, device="cuda")
    b["split"] = torch.empty(8 * n, dtype=torch.float32, device="cuda")
    s = L.DevSystem()
    s.n_part = s.n_src = n
    s.n_list = len(list_idx)
    s.partial_doubles = 0
    s.n_groups, s.n_items, s.n_splits, s.n_crit_max = 1, 1, 0, ni
    for k in ("src", "groups", "list", "items", "counter", "split"):
        setattr(s, k, b[k].data_ptr())
    return s, b


def run_hand(torch, s, ni, precision, tune):
    acc = torch.empty((s.n_part, 3), dtype=torch.float64, device="cuda")
    pot = torch.empty(s.n_part, dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.call("otoo_force", ctypes.byref(s), acc.data_ptr(), pot.data_ptr(), precision, ctypes.byref(tune), st)
    L.call("otoo_check_status", ctypes.byref(s), st)
    return acc[:ni].cpu().numpy(), pot[:ni].cpu().numpy()


def test_compensated_sums_keep_small_terms_after_a_large_one(torch):
    # 64 targets (masses 1e-14) near the origin, a unit mass at distance 1
    # first in the list, then 10^6 masses of 1e-8 on one side (each term
    # below half an FP32 ulp of the running sum; together 0.5% of the
    # potential): a plain FP32 running sum drops all of them, the per-tile
    # sums with Kahan accumulation keep them.  Reference: the FP64 form on
    # the same list.
    rng = np.random.default_rng(32)
    ni, nl = 64, 1_000_000
    tgt = rng.uniform(-1e-3, 1e-3, (ni, 3))
    heavy = np.array([[-1.0, 0.0, 0.0]])
    light = np.column_stack([rng.uniform(1.5, 2.5, nl), rng.uniform(-0.5, 0.5, nl), rng.uniform(-0.5, 0.5, nl)])
    pos = np.vstack([tgt, heavy, light])
    mass = np.concatenate([np.full(ni, 1e-14), [1.0], np.full(nl, 1e-8)]).astype(np.float32)
    lst = np.concatenate([[ni], np.arange(ni), np.arange(ni + 1, ni + 1 + nl)]).astype(np.int32)
    eps = 1e-2
    s, keep = hand_system(torch, pos, mass, lst, ni, eps, (0.0, 0.0, 0.0))
    # 64 targets at two per lane: one lane subset, every lane sums the whole list
    tune = L.Tune(block=128, iblock=2, tile=256, split=1 << 30, ctas_per_sm=0, packed=1)
    a64, p64 = run_hand(torch, s, ni, L.OTOO_FP64, tune)
    a32, p32 = run_hand(torch, s, ni, L.OTOO_FP32K, tune)
    # arithmetic bound of the FP32 form: 2e-6 of sum_j |term_j|, per target
    src = pos[lst]
    m = mass[lst].astype(np.float64)
    sp, sa = np.zeros(ni), np.zeros(ni)
    for i in range(ni):
        d = src - tgt[i]
        r2 = (d * d).sum(1) + eps * eps
        w = np.where(lst == i, 0.0, m)
        sp[i] = (w / np.sqrt(r2)).sum()
        sa[i] = (w * np.sqrt(r2 - eps * eps) / r2 ** 1.5).sum()
    assert np.all(np.abs(p32 - p64) <= 2e-6 * sp)
    assert np.all(np.linalg.norm(a32 - a64, axis=1) <= 2e-6 * sa)
    # a plain FP32 running sum in list order misses the bound by far: after
    # the first (unit) term every later one is below half an ulp and is lost
    d = src - tgt[0]
    terms = np.where(lst == 0, 0.0, m / np.sqrt((d * d).sum(1) + eps * eps)).astype(np.float32)
    assert terms[1:].max() < 0.5 * np.spacing(np.float32(1.0))
    naive = np.float32(0.0)
    for t in terms[:20000]:
        naive = np.float32(naive + t)
    assert float(naive) == float(terms[0])
    dropped = float(terms[1:].sum(dtype=np.float64))
    assert dropped > 1000 * 2e-6 * sp[0]


def test_throughput_probe_kinds(torch):
    # otoo_fma_probe: every kind launches and reports its operation count
    # (resident threads x 8 chains x iters x operations per instruction);
    # an unknown kind is refused
    n = int(L.load().otoo_fma_probe_threads())
    assert n > 0 and n % 256 == 0
    sink = torch.empty(n, dtype=torch.float32, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for kind, per_op in ((0, 2.0), (1, 4.0), (2, 2.0), (3, 1.0)):
        fl = ctypes.c_double(0.0)
        L.call("otoo_fma_probe", 16, kind, sink.data_ptr(), ctypes.byref(fl), st)
        torch.cuda.synchronize()
        ops = fl.value / (8 * 16 * per_op)
        assert ops == int(ops) and 0 < ops <= n and int(ops) % 256 == 0, (kind, fl.value)
    with pytest.raises(L.OtooError) as e:
        L.call("otoo_fma_probe", 16, 4, sink.data_ptr(), ctypes.byref(ctypes.c_double(0.0)), st)
    assert e.value.code == L.OTOO_EINVAL
