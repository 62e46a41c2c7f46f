"""GPU parity of the FP64 LU path (panel, interchanges, substitution, update,
triangular solves) against the CPU oracle, element by element.

Tolerances (FP64, unit roundoff u = 2^-53):
  * pivots: identical on inputs whose smallest relative pivot gap (oracle
    diagnostic) exceeds 1e-10 -- far above the ~n*u perturbation that blocking
    and FMA introduce;
  * packed factors: |LU_gpu - LU_oracle| <= 1e-11 * max|LU| for n <= 1024
    (GEPP forward error ~ n u growth; blocking only reorders sums);
  * exact dyadic products: bit for bit;
  * backward error of the solution: <= 1e-14 (spec bound).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_07174_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _lu_gpu(A, nb=0):
    LU, ipiv, info = api.lu_factor(A.to(DEV), nb=nb)
    torch.cuda.synchronize()
    return LU.cpu().numpy(), ipiv.cpu().numpy(), int(info.item())


@pytest.mark.parametrize("n,nb", [(1, 0), (2, 0), (3, 32), (31, 32), (33, 32), (64, 64), (127, 64),
                                  (129, 64), (257, 96), (300, 64), (700, 256), (1024, 128)])
def test_lu_matches_oracle(n, nb):
    A = inputs.uniform(n, seed=1000 + n)
    An = np.asfortranarray(A.numpy())
    assert oracle.min_pivot_gap(An) > 1e-10
    LUo, ipo, info_o = oracle.getrf(An)
    LUg, ipg, info_g = _lu_gpu(A, nb)
    assert info_g == info_o == 0
    assert np.array_equal(ipg, ipo)
    assert np.abs(LUg - LUo).max() <= 1e-11 * max(1.0, np.abs(LUo).max())


@pytest.mark.parametrize("n,nb", [(5, 32), (64, 32), (300, 64), (777, 256)])
def test_lu_dyadic_exact(n, nb):
    A, L0, U0, perm = inputs.dyadic_lu(n, seed=900 + n)
    LUg, ipg, info = _lu_gpu(A, nb)
    L, U = oracle.unpack_lu(LUg)
    assert info == 0
    assert np.array_equal(L, L0.numpy()) and np.array_equal(U, U0.numpy())
    assert np.array_equal(oracle.perm_from_ipiv(ipg, n), perm.numpy())


def test_config_n512_one_rhs():
    """Plain FP64 LU + one-RHS solve, n = 512, A iid U[-1,1] seed 0, x_true = 1."""
    n = 512
    A = inputs.uniform(n, seed=0)
    b = A @ torch.ones(n, dtype=torch.float64)
    An = np.asfortranarray(A.numpy())
    LUo, ipo, _ = oracle.getrf(An)
    LU, ipiv, info = api.lu_factor(A.to(DEV))
    x = api.lu_solve(LU, ipiv, b.to(DEV))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    assert np.array_equal(ipiv.cpu().numpy(), ipo)
    xo = oracle.getrs(LUo, ipo, b.numpy())[:, 0]
    xg = x.cpu().numpy()
    assert np.abs(xg - xo).max() <= 1e-12
    assert oracle.backward_error(An, xg, b.numpy())[0] <= 1e-14


@pytest.mark.parametrize("n,nrhs", [(65, 1), (300, 3), (513, 16), (200, 21)])
@pytest.mark.parametrize("trans", [False, True])
def test_lu_solve_matches_oracle(n, nrhs, trans):
    A = inputs.uniform(n, seed=n)
    B = inputs.normal((n, nrhs), seed=n + 1)
    An = np.asfortranarray(A.numpy())
    LU, ipiv, info = api.lu_factor(A.to(DEV), nb=64)
    X = api.lu_solve(LU, ipiv, B.to(DEV), trans=trans).cpu().numpy()
    Aop = An.T.copy(order="F") if trans else An
    LUo, ipo, _ = oracle.getrf(Aop)
    Xo = oracle.getrs(LUo, ipo, B.numpy())
    scale = max(1.0, np.abs(Xo).max())
    assert np.abs(X - Xo).max() <= 1e-9 * scale
    assert oracle.backward_error(Aop, X, B.numpy()).max() <= 1e-14


def test_lu_singular_zero_column():
    n, k = 200, 77
    A = inputs.uniform(n, seed=5)
    A[:, k] = 0.0
    LUo, ipo, info_o = oracle.getrf(np.asfortranarray(A.numpy()))
    LUg, ipg, info_g = _lu_gpu(A, 64)
    assert info_o == k + 1
    assert info_g == k + 1
    assert np.array_equal(ipg[:k + 1], ipo[:k + 1])


def test_lu_leading_dimension_padded():
    n, lda = 150, 173
    A = inputs.uniform(n, seed=17)
    store = torch.zeros((lda, n), dtype=torch.float64)
    store[:n] = A
    Ad = store.to(DEV).t().contiguous().t()           # (lda, n) column-major
    Av = Ad[:n]                                        # (n, n) view, strides (1, lda)
    assert Av.stride() == (1, lda)
    LU, ipiv, info = api.lu_factor(Av, nb=64)
    LUo, ipo, _ = oracle.getrf(np.asfortranarray(A.numpy()))
    assert np.array_equal(ipiv.cpu().numpy(), ipo)
    assert np.abs(LU.cpu().numpy() - LUo).max() <= 1e-11 * np.abs(LUo).max()


def test_backward_error_kernel_matches_oracle():
    n, nrhs = 777, 3
    A = inputs.uniform(n, seed=3)
    X = inputs.normal((n, nrhs), seed=4)
    B = A @ X + 1e-9 * inputs.normal((n, nrhs), seed=5)
    beta = api.backward_error(A.to(DEV), X.to(DEV), B.to(DEV)).cpu().numpy()
    beta_o = oracle.backward_error(np.asfortranarray(A.numpy()), X.numpy(), B.numpy())
    # both sides round r = b - A x differently; |d beta| <= 2 gamma_n (Higham 3.5)
    assert np.abs(beta - beta_o).max() <= 2 * n * 2.0 ** -53


@pytest.mark.parametrize("prec,n", [("fp64", 2048), ("fp64", 4224), ("bf16", 1024)])
def test_wait_timeout_reports_status(prec, n):
    """A wait limit of 0 ns makes the inter-CTA waits give up at once: the
    cluster panel (FP64 n = 2048; FP32 in the bf16 case, with the tensor-core
    update after it), the cooperative panel of rows beyond one cluster (FP64
    n = 4224). The call must end with GBLA_INFO_TIMEOUT in info and pivots
    that are all in range; the context must stay usable, and the next
    factorisation (with the limit restored) must be correct."""
    A = inputs.uniform(n, seed=9).to(DEV)
    old = api.get_wait_timeout_ns()
    try:
        api.set_wait_timeout_ns(0)
        if prec == "fp64":
            LU, ipiv, info = api.lu_factor(A, nb=64)
        else:
            LU, ipiv, info = api.lu_factor_mixed(A, prec=prec, nb=128)
        torch.cuda.synchronize()
        v = int(info.item())
        piv = ipiv.cpu().numpy()
    finally:
        api.set_wait_timeout_ns(old)
    assert v == -1000
    assert np.all(piv >= np.arange(1, n + 1)) and np.all(piv <= n)
    # the context still works, and gives the oracle's factorisation
    m = 300
    B = inputs.uniform(m, seed=10)
    LUg, ipg, info_g = _lu_gpu(B, 64)
    LUo, ipo, _ = oracle.getrf(np.asfortranarray(B.numpy()))
    assert info_g == 0
    assert np.array_equal(ipg, ipo)
    assert np.abs(LUg - LUo).max() <= 1e-11 * np.abs(LUo).max()
