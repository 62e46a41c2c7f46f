"""CPU-side checks of the C ABI: the library loads, exports every symbol the
header declares, and rejects invalid arguments before touching the device."""
import ctypes
import os

import pytest

from paper_1511_07174_gb300 import _lib


@pytest.fixture(scope="module")
def lib():
    from paper_1511_07174_gb300 import build
    build.build()
    return _lib.load()


def test_header_symbols_exported(lib):
    syms = _lib.header_symbols()
    assert len(syms) >= 10
    for name in syms:
        assert hasattr(lib, name), name
    # every declared symbol has a ctypes signature in the binding
    assert set(syms) <= set(_lib._SIGS), set(syms) - set(_lib._SIGS)


def test_version_and_status(lib):
    assert b"gbla" in lib.gbla_version()
    assert _lib.status_string(0) == "success"
    assert "workspace" in _lib.status_string(1001)
    assert _lib.status_string(-3) == "invalid argument"


def test_wait_timeout_roundtrip(lib):
    old = lib.gbla_get_wait_timeout_ns()
    lib.gbla_set_wait_timeout_ns(12345)
    assert lib.gbla_get_wait_timeout_ns() == 12345
    lib.gbla_set_wait_timeout_ns(old)


def test_substitution_ctas_roundtrip(lib):
    old = lib.gbla_get_substitution_ctas()
    assert lib.gbla_set_substitution_ctas(-1) == -1
    assert lib.gbla_set_substitution_ctas(24) == 0
    assert lib.gbla_get_substitution_ctas() == 24
    assert lib.gbla_set_substitution_ctas(old) == 0


def test_lookahead_roundtrip(lib):
    old = lib.gbla_get_lookahead()
    assert lib.gbla_set_lookahead(2) == -1
    assert lib.gbla_set_lookahead(1) == 0 and lib.gbla_get_lookahead() == 1
    assert lib.gbla_set_lookahead(old) == 0


def test_invalid_arguments_rejected_on_host(lib):
    v = ctypes.c_void_p(0)
    assert lib.gbla_lu_factor(-1, v, 1, v, v, 0, v, 0, v) == -1
    t = ctypes.c_double(0.0)
    assert lib.gbla_fma_peak(2, 16, ctypes.byref(t), v) == -1
    assert lib.gbla_fma_peak(0, 0, ctypes.byref(t), v) == -2
    assert lib.gbla_fma_peak(0, 16, None, v) == -3
    assert lib.gbla_lu_factor(4, v, 4, v, v, 0, v, 0, v) == -2
    fake = ctypes.c_void_p(256)
    assert lib.gbla_lu_factor(4, fake, 3, fake, fake, 0, fake, 0, v) == -3
    assert lib.gbla_lu_factor(4, fake, 4, fake, fake, 48, fake, 0, v) == -6
    assert lib.gbla_lu_factor(4, fake, 4, fake, fake, 0, v, 0, v) == 1001
    assert lib.gbla_lu_solve(2, 4, 1, fake, 4, fake, fake, 4, fake, fake, 1 << 20, v) == -1
    assert lib.gbla_lu_solve(0, 4, -1, fake, 4, fake, fake, 4, fake, fake, 1 << 20, v) == -3
    assert lib.gbla_lu_factor_mixed(4, fake, 4, fake, 4, fake, fake, 9, 0, fake, 1 << 20, v) == -8
    assert lib.gbla_backward_error(4, 1, fake, 2, fake, 4, fake, 4, fake, fake, 1 << 20, v) == -4
    assert lib.gbla_chol_factor(4, fake, 4, fake, 96, v) == -5      # nb not a multiple of 64
    assert lib.gbla_chol_factor(4, fake, 4, fake, 320, v) == -5
    opts = _lib.GmresirOpts(1e-14, 1e-8, 10, 500, 1)
    st = _lib.GmresirStats()
    assert lib.gbla_gmresir_solve(4, fake, 4, fake, 4, fake, fake, fake, ctypes.byref(opts),
                                  ctypes.byref(st), fake, 1 << 20, v) == -9
    opts = _lib.GmresirOpts(1e-14, 1e-8, 10, 50, -1)       # negative restart count
    assert lib.gbla_gmresir_solve(4, fake, 4, fake, 4, fake, fake, fake, ctypes.byref(opts),
                                  ctypes.byref(st), fake, 1 << 20, v) == -9
    opts = _lib.GmresirOpts(1e-14, 1e-8, 10, 50, 2)
    sts = (_lib.GmresirStats * 3)()
    nrhs = lib.gbla_gmresir_solve_nrhs
    assert nrhs(4, -1, fake, 4, fake, 4, fake, fake, 4, fake, 4, ctypes.byref(opts), sts, fake,
                1 << 20, v) == -2
    assert nrhs(4, 3, fake, 4, fake, 4, fake, fake, 3, fake, 4, ctypes.byref(opts), sts, fake,
                1 << 20, v) == -9
    assert nrhs(4, 3, fake, 4, fake, 4, fake, fake, 4, fake, 4, ctypes.byref(opts), None, fake,
                1 << 20, v) == -13
    assert nrhs(4, 3, fake, 4, fake, 4, fake, fake, 4, fake, 4, ctypes.byref(opts), sts, v,
                1 << 20, v) == 1001
    # no right-hand sides: nothing to do, nothing touched
    assert nrhs(4, 0, fake, 4, fake, 4, fake, v, 4, v, 4, ctypes.byref(opts), None, fake,
                1 << 20, v) == 0


def test_workspace_sizes(lib):
    assert lib.gbla_lu_factor_workspace(1000, 0) > 0
    assert lib.gbla_lu_factor_workspace(1000, 40) == 0          # invalid nb
    assert lib.gbla_lu_factor_mixed_workspace(1000, 256, 3) > lib.gbla_lu_factor_workspace(1000, 256)
    assert lib.gbla_gmresir_workspace(1000, 50) >= 1000 * 51 * 8
    assert lib.gbla_lu_solve_workspace(100, 4) >= 100 * 4 * 8


def test_batched_arguments_rejected_on_host(lib):
    v = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(256)
    ws = lib.gbla_chol_batched_workspace(8)
    assert ws > 0 and lib.gbla_lu_batched_workspace(8) > 0
    assert lib.gbla_chol_batched_workspace(-1) == 0
    # batch < 0; missing sizes, matrices, leading dimensions; rhs without B
    assert lib.gbla_chol_solve_batched(-1, v, v, v, v, v, v, v, v, 0, 0, 0, fake, ws, v) == -1
    assert lib.gbla_chol_solve_batched(2, v, fake, fake, v, v, v, v, v, 0, 0, 0, fake, ws, v) == -2
    assert lib.gbla_chol_solve_batched(2, fake, v, fake, v, v, v, v, v, 0, 0, 0, fake, ws, v) == -3
    assert lib.gbla_chol_solve_batched(2, fake, fake, v, v, v, v, v, v, 0, 0, 0, fake, ws, v) == -4
    assert lib.gbla_chol_solve_batched_f32(2, fake, fake, fake, fake, v, fake, v, v, 0, 0, 0, fake, ws, v) == -6
    # launch-shape knobs and workspace
    assert lib.gbla_chol_solve_batched(2, fake, fake, fake, v, v, v, v, v, -1, 0, 0, fake, ws, v) == -10
    assert lib.gbla_chol_solve_batched(2, fake, fake, fake, v, v, v, v, v, 0, 48, 0, fake, ws, v) == -11
    assert lib.gbla_chol_solve_batched(2, fake, fake, fake, v, v, v, v, v, 0, 0, 33, fake, ws, v) == -12
    assert lib.gbla_chol_solve_batched(2, fake, fake, fake, v, v, v, v, v, 0, 0, 0, v, ws, v) == 1001
    # an empty batch is a no-op that touches nothing
    assert lib.gbla_chol_solve_batched(0, v, v, v, v, v, v, v, v, 0, 0, 0, fake, ws, v) == 0
    assert lib.gbla_lu_solve_batched(-1, v, v, v, v, v, v, v, v, v, 0, 0, 0, fake, ws, v) == -1
    assert lib.gbla_lu_solve_batched(2, fake, fake, fake, v, v, v, v, v, v, 0, 0, 0, fake, ws, v) == -5


def test_krylov_arguments_rejected_on_host(lib):
    v = ctypes.c_void_p(0)
    fake = ctypes.c_void_p(256)
    ws = lib.gbla_krylov_workspace(16, 8)
    assert ws > 0 and lib.gbla_krylov_workspace(16, 0) == 0 and lib.gbla_krylov_workspace(-1, 8) == 0
    st = _lib.KrylovStats()
    ok = _lib.KrylovOpts(1e-10, 10, 8)
    for fn in (lib.gbla_gmres_solve, lib.gbla_bicgstab_solve):
        assert fn(-1, fake, 1, fake, fake, v, 1, v, ctypes.byref(ok), ctypes.byref(st), fake, ws, v) == -1
        assert fn(4, fake, 3, fake, fake, v, 1, v, ctypes.byref(ok), ctypes.byref(st), fake, ws, v) == -3
        # factors without pivots (or the reverse)
        assert fn(4, fake, 4, fake, fake, fake, 4, v, ctypes.byref(ok), ctypes.byref(st), fake, ws, v) == -6
        bad = _lib.KrylovOpts(-1.0, 10, 8)
        assert fn(4, fake, 4, fake, fake, v, 1, v, ctypes.byref(bad), ctypes.byref(st), fake, ws, v) == -9
        bad = _lib.KrylovOpts(1e-10, 10, 129)
        assert fn(4, fake, 4, fake, fake, v, 1, v, ctypes.byref(bad), ctypes.byref(st), fake, ws, v) == -9
        assert fn(4, fake, 4, fake, fake, v, 1, v, ctypes.byref(ok), None, fake, ws, v) == -10
        assert fn(4, fake, 4, fake, fake, v, 1, v, ctypes.byref(ok), ctypes.byref(st), v, ws, v) == 1001
        # n = 0: converged, nothing touched
        assert fn(0, v, 1, v, v, v, 1, v, ctypes.byref(ok), ctypes.byref(st), fake, ws, v) == 0
        assert st.converged == 1
