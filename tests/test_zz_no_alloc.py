"""gbla_lu_factor_static: the LU factor entry point for callers that cannot
allocate device memory (its scratch is a fixed array in the library's device
image). Called through the C ABI; its output must match gbla_lu_factor's on
the same inputs, on two calls in a row (the second call reuses the array the
first one left behind). Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1511_07174_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _static_factor(A, nb, expect_rc=0):
    n = A.shape[0]
    LU = api.colmajor(A.to(DEV), torch.float64, copy=True)
    ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=DEV)
    info = torch.full((1,), 7, dtype=torch.int32, device=DEV)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _lib.load().gbla_lu_factor_static(n, ctypes.c_void_p(LU.data_ptr()), LU.stride(1),
                                           ctypes.c_void_p(ipiv.data_ptr()),
                                           ctypes.c_void_p(info.data_ptr()), nb, stream)
    assert rc == expect_rc, (rc, _lib.load().gbla_last_error())
    torch.cuda.synchronize()
    return LU.cpu().numpy(), ipiv[:n].cpu().numpy(), int(info.item())


@pytest.mark.parametrize("seed", [0])
def test_static_matches_workspace_entry_twice(seed):
    for n, nb in [(700, 128), (1000, 256)]:       # two calls in a row
        A = inputs.uniform(n, seed=seed + n)
        LUs, ips, infos = _static_factor(A, nb)
        LUw, ipw, infow = api.lu_factor(A.to(DEV), nb=nb)
        torch.cuda.synchronize()
        assert infos == int(infow.item()) == 0
        assert np.array_equal(ips, ipw.cpu().numpy())
        LUw = LUw.cpu().numpy()
        assert np.abs(LUs - LUw).max() <= 1e-11 * np.abs(LUw).max()


def test_static_rejects_bad_arguments():
    L = _lib.load()
    v = ctypes.c_void_p(0)
    assert L.gbla_lu_factor_static(-1, v, 1, v, v, 0, v) == -1
    assert L.gbla_lu_factor_static(8, ctypes.c_void_p(256), 8, ctypes.c_void_p(256),
                                   ctypes.c_void_p(256), 40, v) == -6


def test_static_after_a_call_that_gave_up():
    """The shared array is cleared by every call, so slot words left by a call
    whose waits gave up part way (wait limit 0: info = GBLA_INFO_TIMEOUT) cannot
    be mistaken for fresh ones by the next call: it must match gbla_lu_factor."""
    n, nb = 1000, 128
    old = api.get_wait_timeout_ns()
    try:
        api.set_wait_timeout_ns(0)
        _, _, info0 = _static_factor(inputs.uniform(n, seed=41), nb)
    finally:
        api.set_wait_timeout_ns(old)
    assert info0 == -1000
    A = inputs.uniform(n, seed=42)
    LUs, ips, infos = _static_factor(A, nb)
    LUw, ipw, infow = api.lu_factor(A.to(DEV), nb=nb)
    torch.cuda.synchronize()
    assert infos == int(infow.item()) == 0
    assert np.array_equal(ips, ipw.cpu().numpy())
    LUw = LUw.cpu().numpy()
    assert np.abs(LUs - LUw).max() <= 1e-11 * np.abs(LUw).max()
