"""Host-library checks that need no GPU: the host half of the C ABI built
with the address and undefined-behaviour sanitizers and exercised by a
driver of its own (tests/host_check/driver.cpp), and allocation failure
turned into OTOO_ENOMEM (the process's address space capped below what a
tree needs)."""
import os
import shutil
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_host_library_under_address_and_ub_sanitizers(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    from paper_1206_1199_gb300 import build
    exe = str(tmp_path / "driver")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined", "-fopenmp",
           "-ffp-contract=off", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(build._cuda_home(), "include"),  # NVTX (header-only)
           os.path.join(ROOT, "tests", "host_check", "driver.cpp"),
           os.path.join(ROOT, "paper_1206_1199_gb300", "csrc", "host", "tree.cpp"), "-o", exe, "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime not available: " + r.stderr[-200:])
    assert r.returncode == 0, r.stderr[-2000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1", OMP_NUM_THREADS="4")
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, (r.stdout[-1000:], r.stderr[-4000:])
    assert "runtime error" not in r.stderr and "ERROR: AddressSanitizer" not in r.stderr, r.stderr[-4000:]
    assert "0 failed" in r.stdout


def test_allocation_failure_is_enomem():
    script = textwrap.dedent("""
        import resource, sys
        import numpy as np
        sys.path.insert(0, %r)
        from paper_1206_1199_gb300 import _lib as L, system as S
        L.load()
        n = 4000000
        pos = np.random.default_rng(1).random((n, 3))
        mass = np.full(n, 1.0 / n, np.float32)
        S.Tree(pos[:1000], mass[:1000])       # the library works before the cap
        page = resource.getpagesize()
        vm = int(open("/proc/self/statm").read().split()[0]) * page
        resource.setrlimit(resource.RLIMIT_AS, (vm + (48 << 20), resource.RLIM_INFINITY))
        try:
            S.Tree(pos, mass)                   # the tree's host arrays need far more
        except L.OtooError as e:
            print("code", e.code)
            sys.exit(0)
        print("no error")
    """ % ROOT)
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", script], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    from paper_1206_1199_gb300 import _lib as L
    assert r.stdout.strip().endswith("code %d" % L.OTOO_ENOMEM), r.stdout
