"""The allocation-free force entry point (otoo_force_static), called through
the C ABI, against the allocating one (otoo_force) on the same device inputs.

Callers that cannot allocate device memory (their GPU memory is owned by
another allocator, or their loop must not enter the CUDA runtime's allocator) use
otoo_force_static: its scratch is a library-held device array.  This file is
collected last so that a failure here leaves every other test already run;
it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest

from paper_1206_1199_gb300 import _lib as L
from paper_1206_1199_gb300 import ic, system as S

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)


def static_force(dev, precision, tune):
    import torch
    n = dev.lists.n_part
    acc = torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda")
    pot = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    L.call("otoo_force_static", ctypes.byref(dev.struct), dev.plan.partial_doubles, acc.data_ptr(), pot.data_ptr(),
           int(precision), ctypes.byref(tune), ctypes.c_void_p(st.cuda_stream))
    # the status word of the call lives in the library's array too
    L.call("otoo_force_static_status", ctypes.c_void_p(st.cuda_stream))
    return acc.cpu().numpy(), pot.cpu().numpy()


@pytest.mark.parametrize("precision", [L.OTOO_FP32K, L.OTOO_FP64])
def test_static_scratch_matches_allocating_entry_point(precision):
    import torch  # noqa: F401
    L.load()
    pos, mass = ic.plummer(10000, 31)
    tune = L.default_tune(64)
    tune.split = 1000  # long lists are cut: the chunk partials live in the static array too
    tree, lists, plan = S.build_system(pos, mass, 0.5, 64, 1e-2, tune=tune)
    assert plan.n_splits > 0
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    ref_a, ref_p = S.force(dev, precision=precision, tune=tune)
    ref_a, ref_p = ref_a.cpu().numpy(), ref_p.cpu().numpy()
    for _ in range(2):  # two calls in a row share (and reuse) the array
        a, p = static_force(dev, precision, tune)
        assert np.all(np.isfinite(a)) and np.all(np.isfinite(p))
        d = rel(a, ref_a)
        dp = np.abs(p - ref_p) / np.abs(ref_p)
        if precision == L.OTOO_FP64:
            assert d.max() <= 1e-10 and dp.max() <= 1e-10
        else:
            assert np.sqrt(np.mean(d * d)) <= 2e-6 and d.max() <= 2e-4 and dp.max() <= 1e-5


def test_static_scratch_rejects_oversized_step():
    import torch  # noqa: F401
    L.load()
    pos, mass = ic.plummer(2000, 32)
    tree, lists, plan = S.build_system(pos, mass, 0.5, 64, 1e-2)
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    cap = int(L.load().otoo_force_static_capacity())
    with pytest.raises(L.OtooError) as e:
        L.call("otoo_force_static", ctypes.byref(dev.struct), cap // 8, dev.bufs["partial"].data_ptr(),
               dev.bufs["partial"].data_ptr(), L.OTOO_FP32K, ctypes.byref(plan.tune), None)
    assert e.value.code == L.OTOO_EINVAL and "scratch" in str(e.value)


def test_static_status_reports_slots_past_the_partial_part():
    # a partial part smaller than the plan needs: the items and splits whose
    # slots reach past it are skipped, and otoo_force_static_status says so
    import torch
    L.load()
    pos, mass = ic.plummer(10000, 31)
    tune = L.default_tune(64)
    tune.split = 1000
    tree, lists, plan = S.build_system(pos, mass, 0.5, 64, 1e-2, tune=tune)
    assert plan.partial_doubles > 4 * plan.n_crit_max
    dev = S.DeviceSystem.upload(lists, plan, "cuda")
    n = lists.n_part
    acc = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    pot = torch.zeros((n,), dtype=torch.float64, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.call("otoo_force_static", ctypes.byref(dev.struct), 4 * plan.n_crit_max, acc.data_ptr(), pot.data_ptr(),
           L.OTOO_FP32K, ctypes.byref(tune), st)
    with pytest.raises(L.OtooError) as e:
        L.call("otoo_force_static_status", st)
    assert e.value.code == L.OTOO_EDEVICE
    # the next call clears the status word
    a, p = static_force(dev, L.OTOO_FP32K, tune)
    assert np.all(np.isfinite(a))
