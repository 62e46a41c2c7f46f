"""GPU parity of the FP64 Cholesky path against the CPU oracle.

Tolerances (u = 2^-53): L within 1e-12 * max|L| of the oracle's (Cholesky is
backward stable and ||L|| ~ ||A||^(1/2); blocking only reorders sums); exact
integer L L^t recovered bit for bit; the upper triangle is never touched;
solution backward error <= 1e-14; the first non-positive leading minor
reported as the oracle reports it.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_07174_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("n", [1, 5, 31, 33, 63, 64, 65, 130, 300, 1000])
@pytest.mark.parametrize("nb", [64, 128, 192, 256])
def test_chol_matches_oracle(n, nb):
    """Every outer block width the tuner can pick: one block, several blocks and
    ragged last blocks (n = 130, 300, 1000 against nb = 128 .. 256)."""
    A = inputs.spd(n, seed=n)
    An = np.asfortranarray(A.numpy())
    Lo, info_o = oracle.potrf(An)
    F, info = api.chol_factor(A.to(DEV), nb=nb)
    torch.cuda.synchronize()
    Fg = F.cpu().numpy()
    assert int(info.item()) == info_o == 0
    assert np.abs(np.tril(Fg) - np.tril(Lo)).max() <= 1e-12 * np.abs(np.tril(Lo)).max()
    assert np.array_equal(np.triu(Fg, 1), np.triu(An, 1))


@pytest.mark.parametrize("n", [3, 64, 100, 257, 600])
@pytest.mark.parametrize("nb", [64, 192])
def test_chol_dyadic_exact(n, nb):
    A, L0 = inputs.dyadic_chol(n, seed=700 + n)
    F, info = api.chol_factor(A.to(DEV), nb=nb)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert np.array_equal(np.tril(F.cpu().numpy()), L0.numpy())


@pytest.mark.parametrize("n,k", [(10, 3), (200, 0), (200, 64), (200, 150), (600, 300)])
@pytest.mark.parametrize("nb", [64, 256])
def test_chol_not_spd(n, k, nb):
    A = inputs.spd(n, seed=11).numpy()
    A[k, k] = -1.0
    _, info_o = oracle.potrf(np.asfortranarray(A))
    F, info = api.chol_factor(torch.from_numpy(A).to(DEV), nb=nb)
    torch.cuda.synchronize()
    assert info_o == k + 1
    assert int(info.item()) == k + 1


@pytest.mark.parametrize("n,nrhs", [(65, 1), (500, 16), (300, 21)])
def test_chol_solve(n, nrhs):
    A = inputs.spd(n, seed=2)
    B = inputs.normal((n, nrhs), seed=3)
    F, info = api.chol_factor(A.to(DEV))
    X = api.chol_solve(F, B.to(DEV)).cpu().numpy()
    An = np.asfortranarray(A.numpy())
    Lo, _ = oracle.potrf(An)
    Xo = oracle.potrs(Lo, B.numpy())
    assert np.abs(X - Xo).max() <= 1e-10 * np.abs(Xo).max()
    assert oracle.backward_error(An, X, B.numpy()).max() <= 1e-14


@pytest.mark.slow
def test_chol_full_size_n8192():
    """n = 8192, A = B B^t / n + I: backward error of a 16-RHS solve and sampled
    rows of A - L L^t, both with the oracle's plain FP64 arithmetic."""
    n, nrhs = 8192, 16
    A = inputs.spd(n, seed=2, device=DEV)
    X_true = inputs.normal((n, nrhs), seed=3, device=DEV)
    B = A @ X_true
    F, info = api.chol_factor(A)
    X = api.chol_solve(F, B)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    An = np.asfortranarray(A.cpu().numpy())
    beta = oracle.backward_error(An, X.cpu().numpy(), B.cpu().numpy())
    assert beta.max() <= 1e-14
    L = np.tril(F.cpu().numpy())
    rows = np.random.default_rng(0).choice(n, 16, replace=False)
    R = An[rows] - L[rows] @ L.T
    assert np.abs(R).max() <= 64 * n * 2.0 ** -53 * np.abs(An).max()


def test_block_size_tuners():
    """tune_lu_nb / tune_chol_nb time their candidates on a matrix of the given
    order and return one of them; the factorisation with the chosen block size
    still matches the oracle."""
    n = 1024
    nb = api.tune_lu_nb(n, use_cache=False)
    assert nb in (64, 96, 128, 192, 256)
    nbc = api.tune_chol_nb(n, use_cache=False)
    assert nbc in (64, 128, 192, 256)
    A = inputs.spd(n, seed=5)
    F, info = api.chol_factor(A.to(DEV), nb=nbc)
    Lo, _ = oracle.potrf(np.asfortranarray(A.numpy()))
    assert int(info.item()) == 0
    assert np.abs(np.tril(F.cpu().numpy()) - np.tril(Lo)).max() <= 1e-12 * np.abs(np.tril(Lo)).max()
