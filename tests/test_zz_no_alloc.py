"""The allocation-free ORAS entry point against the regular one.

mwi_oras_apply_device_noalloc serves callers that cannot call cudaMalloc
while they run (a process whose device memory belongs to a pool allocator, or
a latency-critical loop that must not pay cudaMalloc's implicit device
synchronisation).  It takes its scratch from a fixed 32 MiB device array
instead of allocating.  Here it must give the same result as
mwi_oras_apply_device, through the C ABI, on two calls in a row (the shared
scratch keeps the previous call's contents), in the FP64 and the mixed path:
bit for bit, since both run the same kernels on the same inputs.  Once the
first call has looked up the scratch array's address, a call makes no device
allocation (the library's cudaMalloc counter does not move).  A problem whose
scratch would not fit is rejected.

This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""

import ctypes as C

import numpy as np
import pytest

from oracle import dd
from tests._helpers import FREQ, chamber_case, rel_err

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# the ORAS-apply tolerances of tests/test_gpu_parity.py
TOL = {0: 1e-10, 1: 2e-5}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1607_02573_gb300 import mwi
    return mwi


@pytest.mark.parametrize("precision", [0, 1])
def test_noalloc_matches_regular_entry_point(lib, precision):
    mesh, eps, tx, rx = chamber_case(12, 11)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    part = dd.rcb_partition(mesh.xyz, mesh.tet, 6)
    P = lib.Problem(M, eps, FREQ, n_sub=6, part=part, precision=precision)
    rng = np.random.default_rng(7 + precision)
    m = 3
    for call in range(2):
        X = rng.standard_normal((M.ndof, m)) + 1j * rng.standard_normal((M.ndof, m))
        x = torch.from_numpy(X).cuda()
        y_ref = torch.empty_like(x)
        y_new = torch.full_like(x, float("nan"))
        lib.check(lib.mwi_oras_apply_device(P.h, C.c_void_p(x.data_ptr()), C.c_void_p(y_ref.data_ptr()), m))
        torch.cuda.synchronize()
        n_alloc = lib.mwi_device_alloc_count()
        lib.check(lib.mwi_oras_apply_device_noalloc(P.h, C.c_void_p(x.data_ptr()), C.c_void_p(y_new.data_ptr()),
                                                    m))
        torch.cuda.synchronize()
        if call > 0:
            assert lib.mwi_device_alloc_count() == n_alloc, f"call {call}: the library allocated device memory"
        a = y_new.cpu().numpy()
        b = y_ref.cpu().numpy()
        assert np.all(np.isfinite(a)), f"call {call}: non-finite output"
        assert rel_err(a, b) <= TOL[precision], f"call {call}"
        assert np.array_equal(a, b), f"call {call}: not bit for bit"
    P.close()
    M.close()


def test_noalloc_rejects_oversized_scratch(lib):
    mesh, eps, tx, rx = chamber_case(12, 11)
    M = lib.Mesh(mesh.xyz, mesh.tet, mesh.bface_tag)
    P = lib.Problem(M, eps, FREQ, n_sub=6)
    m = 2048  # (local + update rows) * m complex doubles is far beyond 32 MiB
    x = torch.zeros((M.ndof, m), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    st = lib.mwi_oras_apply_device_noalloc(P.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), m)
    assert st == lib.MWI_EINVAL
    assert b"scratch" in lib.mwi_last_error()
    P.close()
    M.close()
