"""Batched LU (and Cholesky) + solve (one persistent launch) against the oracle, system by system.

FP64: pivots identical (tie-free inputs), factors within 1e-11 * max|LU|,
solutions within 1e-10 relative of the oracle's and backward error <= 1e-14.
FP32: pivots identical where the oracle's pivot gap exceeds 1e-4 (FP32
rounding can reorder closer candidates), backward error (computed in FP64 on
the FP32 solution) <= 64 n u32.
Both the shared-memory path (small n) and the in-place global-memory path
(n above the shared-memory limit) are covered, with n = 1 and ragged sizes;
a CUDA-graph replay must reproduce the eager results bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_07174_gb300 import inputs
from paper_1511_07174_gb300.batched import BatchedLU

pytestmark = pytest.mark.gpu


def _mixed_batch(seed, count=40):
    g = torch.Generator().manual_seed(seed)
    sizes = [1, 2, 17, 255, 256, 300] + torch.randint(3, 260, (count - 6,), generator=g).tolist()
    As, Bs = [], []
    for n in sizes:
        As.append(torch.rand((n, n), generator=g, dtype=torch.float64) * 2 - 1)
        Bs.append(torch.randn((n, int(torch.randint(1, 5, (1,), generator=g))), generator=g,
                              dtype=torch.float64))
    return As, Bs


def test_batched_fp64_matches_oracle():
    As, Bs = _mixed_batch(1)
    bl = BatchedLU(As, Bs, dtype=torch.float64)
    bl.restore()
    bl.run()
    torch.cuda.synchronize()
    res, info = bl.results()
    for (LU, piv, X), A, B, inf in zip(res, As, Bs, info.tolist()):
        An = np.asfortranarray(A.numpy())
        LUo, ipo, info_o = oracle.getrf(An)
        assert inf == info_o == 0
        if oracle.min_pivot_gap(An) > 1e-10:
            assert np.array_equal(piv.numpy(), ipo)
            assert np.abs(LU.numpy() - LUo).max() <= 1e-11 * max(1.0, np.abs(LUo).max())
        Xo = oracle.getrs(LUo, ipo, B.numpy())
        assert np.abs(X.numpy() - Xo).max() <= 1e-10 * max(1.0, np.abs(Xo).max()) * A.shape[0]
        assert oracle.backward_error(An, X.numpy(), B.numpy()).max() <= 1e-14


def test_batched_fp32_matches_oracle():
    As, Bs = _mixed_batch(2)
    bl = BatchedLU(As, Bs, dtype=torch.float32)
    bl.restore()
    bl.run()
    torch.cuda.synchronize()
    res, info = bl.results()
    for (LU, piv, X), A, B in zip(res, As, Bs):
        n = A.shape[0]
        A32 = A.to(torch.float32).to(torch.float64).numpy()
        An = np.asfortranarray(A32)
        LUo, ipo, _ = oracle.getrf(An)
        if oracle.min_pivot_gap(An) > 1e-4:
            assert np.array_equal(piv.numpy(), ipo)
        B32 = B.to(torch.float32).to(torch.float64).numpy()
        beta = oracle.backward_error(An, X.to(torch.float64).numpy(), B32).max()
        assert beta <= 64 * n * 2.0 ** -24


def test_batched_graph_replay_and_singular():
    As, Bs = _mixed_batch(3, count=12)
    As[4][:, 2] = 0.0            # singular: zero column -> info = 3
    bl = BatchedLU(As, Bs, dtype=torch.float64)
    bl.restore()
    bl.run()
    torch.cuda.synchronize()
    eagerA, eagerB = bl.A.clone(), bl.B.clone()
    info_e = bl.info.clone()
    bl.capture()
    bl.replay()
    torch.cuda.synchronize()
    # bit-identical (the singular system's solution holds inf / NaN on both runs)
    torch.testing.assert_close(bl.A, eagerA, rtol=0, atol=0, equal_nan=True)
    torch.testing.assert_close(bl.B, eagerB, rtol=0, atol=0, equal_nan=True)
    assert int(info_e[4]) == 3 and int(bl.info[4]) == 3


@pytest.mark.slow
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_4096_uneven(dtype):
    """4096 systems, n_i uniform in [16, 256], A_i iid U[-1,1] + n_i I, 1-4 RHS."""
    sizes, nrhs, As, Bs, Xs = inputs.batched(4096, seed=7)
    bl = BatchedLU(As, Bs, dtype=dtype)
    bl.autotune(use_cache=False)
    bl.capture()
    bl.replay()
    torch.cuda.synchronize()
    res, info = bl.results()
    assert int(info.abs().sum()) == 0
    tol = 1e-14 if dtype == torch.float64 else None
    worst = 0.0
    for (LU, piv, X), A, B in zip(res, As, Bs):
        Ad = A.to(dtype).to(torch.float64).numpy()
        Bd = B.to(dtype).to(torch.float64).numpy()
        beta = oracle.backward_error(np.asfortranarray(Ad), X.to(torch.float64).numpy(), Bd).max()
        lim = tol if tol is not None else 64 * A.shape[0] * 2.0 ** -24
        worst = max(worst, beta / lim)
        # diagonally dominant: partial pivoting keeps the diagonal
        assert np.array_equal(piv.numpy(), np.arange(1, A.shape[0] + 1))
    assert worst <= 1.0


# ------------------------------------------------------------------ Cholesky
def _spd_batch(seed, count=30):
    g = torch.Generator().manual_seed(seed)
    sizes = [1, 2, 17, 255, 256, 300] + torch.randint(3, 260, (count - 6,), generator=g).tolist()
    As, Bs = [], []
    for n in sizes:
        Bm = torch.randn((n, n), generator=g, dtype=torch.float64)
        As.append(Bm @ Bm.t() / n + torch.eye(n, dtype=torch.float64))
        Bs.append(torch.randn((n, int(torch.randint(1, 5, (1,), generator=g))), generator=g,
                              dtype=torch.float64))
    return As, Bs


def test_batched_chol_fp64_matches_oracle():
    """L within 1e-12 max|L| of the oracle's, strict upper triangle untouched,
    solutions within 1e-10 relative and backward error <= 1e-14 (shared-memory
    and in-place paths, n = 1 and ragged sizes)."""
    As, Bs = _spd_batch(11)
    bl = BatchedLU(As, Bs, dtype=torch.float64, method="chol")
    bl.restore()
    bl.run()
    torch.cuda.synchronize()
    res, info = bl.results()
    for (Lf, piv, X), A, B, inf in zip(res, As, Bs, info.tolist()):
        An = np.asfortranarray(A.numpy())
        Lo, info_o = oracle.potrf(An)
        assert inf == info_o == 0 and piv is None
        Lg = Lf.numpy()
        assert np.abs(np.tril(Lg) - np.tril(Lo)).max() <= 1e-12 * max(1.0, np.abs(np.tril(Lo)).max())
        assert np.array_equal(np.triu(Lg, 1), np.triu(A.numpy(), 1))
        Xo = oracle.potrs(Lo, B.numpy())
        assert np.abs(X.numpy() - Xo).max() <= 1e-10 * max(1.0, np.abs(Xo).max())
        assert oracle.backward_error(An, X.numpy(), B.numpy()).max() <= 1e-14


def test_batched_chol_fp32_and_not_spd():
    """FP32: backward error (FP64 on the FP32 solution) <= 64 n u32; a system
    whose third leading minor is negative reports info = 3 and keeps its
    right-hand sides; the others are unaffected; a graph replay reproduces
    the eager run bit for bit."""
    As, Bs = _spd_batch(12, count=12)
    bad = As[5].clone()
    bad[2, 2] = -1.0
    As[5] = bad
    bl = BatchedLU(As, Bs, dtype=torch.float32, method="chol")
    bl.restore()
    bl.run()
    torch.cuda.synchronize()
    eagerA, eagerB, info_e = bl.A.clone(), bl.B.clone(), bl.info.clone()
    res, info = bl.results()
    for i, ((Lf, piv, X), A, B) in enumerate(zip(res, As, Bs)):
        n = A.shape[0]
        A32 = A.to(torch.float32).to(torch.float64).numpy()
        B32 = B.to(torch.float32)
        _, info_o = oracle.potrf(np.asfortranarray(A32))
        assert int(info[i]) == info_o
        if i == 5:
            assert info_o == 3
            assert torch.equal(X, B32)
            continue
        beta = oracle.backward_error(np.asfortranarray(A32), X.to(torch.float64).numpy(),
                                     B32.to(torch.float64).numpy()).max()
        assert beta <= 64 * n * 2.0 ** -24
    bl.capture()
    bl.replay()
    torch.cuda.synchronize()
    torch.testing.assert_close(bl.A, eagerA, rtol=0, atol=0, equal_nan=True)
    torch.testing.assert_close(bl.B, eagerB, rtol=0, atol=0, equal_nan=True)
    assert torch.equal(bl.info, info_e)


@pytest.mark.parametrize("method", ["lu", "chol"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_batched_factor_then_solve(method, dtype):
    """Factor-only launch, then solve-only launches with the stored factors: the
    first right-hand sides give exactly the fused launch's solutions (same
    operations in the same order), and a second set of right-hand sides is
    solved from the same factors (checked against the oracle in FP64)."""
    As, Bs = _mixed_batch(11, count=24)
    if method == "chol":
        As = [(A.t() @ A) / A.shape[0] + torch.eye(A.shape[0], dtype=torch.float64) for A in As]
    fused = BatchedLU(As, Bs, dtype=dtype, method=method)
    fused.restore()
    fused.run()
    torch.cuda.synchronize()
    res_f, info_f = fused.results()
    split = BatchedLU(As, Bs, dtype=dtype, method=method)
    split.restore()
    split.factor()
    split.solve()
    torch.cuda.synchronize()
    res_s, info_s = split.results()
    assert torch.equal(info_f, info_s)
    for (LUf, pf, Xf), (LUs, ps, Xs) in zip(res_f, res_s):
        assert torch.equal(LUf, LUs) and torch.equal(Xf, Xs)
        if method == "lu":
            assert torch.equal(pf, ps)
    g = torch.Generator().manual_seed(12)
    B2 = [torch.randn(B.shape, generator=g, dtype=torch.float64) for B in Bs]
    split.solve(B2)
    torch.cuda.synchronize()
    res2, _ = split.results()
    tol = 1e-14 if dtype == torch.float64 else 64 * 2.0 ** -24
    for (_, _, X), A, B in zip(res2, As, B2):
        Ad = np.asfortranarray(A.to(dtype).to(torch.float64).numpy())
        n = A.shape[0]
        beta = oracle.backward_error(Ad, X.to(torch.float64).numpy(), B.to(dtype).to(torch.float64).numpy())
        assert beta.max() <= tol * (1 if dtype == torch.float64 else n)
