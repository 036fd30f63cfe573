"""Failure detection of the tensor-core z solve without a GPU fault: its waits on MMA
completion and on the bulk copy of the matrices are bounded (tc_ptx.cuh, mbar_wait).  A
kernel waits on an mbarrier that nothing arrives at, with a 20 ms limit: the wait gives up,
the kernel returns, and the context stays usable; with the phase completed the same wait
succeeds at once.  The test kernel (tests/tc_wait_selftest.cu) is built here with the
library's flags."""
import ctypes as ct
import subprocess
import time
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu

HERE = Path(__file__).resolve().parent


@pytest.fixture(scope="module")
def selftest(tmp_path_factory):
    from paper_2104_00350_gb300 import build
    so = tmp_path_factory.mktemp("tcwait") / "libtcwait.so"
    cmd = [build.nvcc(), "-O3", "-std=c++17", *build.ARCH, "-Xcompiler", "-fPIC", "-shared",
           "-o", str(so), str(HERE / "tc_wait_selftest.cu")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ct.CDLL(str(so))
    lib.tc_wait_selftest.argtypes = [ct.c_ulonglong, ct.c_int, ct.POINTER(ct.c_int)]
    lib.tc_wait_selftest.restype = ct.c_int
    return lib


def test_wait_on_an_unset_barrier_gives_up(selftest):
    res = ct.c_int(0)
    t0 = time.perf_counter()
    err = selftest.tc_wait_selftest(20_000_000, 0, ct.byref(res))
    dt = time.perf_counter() - t0
    assert err == 0 and res.value == 2
    assert 0.02 <= dt < 5.0, dt
    res2 = ct.c_int(0)
    assert selftest.tc_wait_selftest(20_000_000, 1, ct.byref(res2)) == 0 and res2.value == 1
    import torch
    x = torch.ones(4, device="cuda")
    assert float((x + 1).sum()) == 8.0
