"""GPU parity of the mixed-precision Cholesky (FP32 arithmetic, trailing update
on the tensor cores for the lower tiles only, or FP32 SIMT) and of its GMRES
refinement, against the oracle's low-precision Cholesky (oracle/mixed.py).

* exact integer factors: every precision recovers L bit for bit, and the
  strict upper triangle of F holds L^t;
* random SPD inputs, entry by entry against the oracle (no pivoting, so the
  two eliminations take the same steps): the panel and substitution differ by
  at most one FP32 rounding per operation (FP32 arithmetic against FP64
  rounded to FP32), the update products take the same rounded operands and
  differ in the FP32 accumulation order and, when a one-ulp difference moves
  an operand across a rounding boundary, by one unit of the update format:
  |F - F_oracle| <= n * u * max(|L||L^t|), u as in the LU tests;
* GMRES-IR reaches backward error <= 1e-14 (oracle FP64 matvec) where
  kappa * u_p <= 10, for one and several right-hand sides;
* a non-positive leading minor is reported as the oracle reports it.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import mixed as M
from paper_1511_07174_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
PRECS = ["fp32", "tf32", "bf16", "fp16", "fp16x3", "bf16x3"]
UNIT = {"fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11,
        "fp16x3": 2.0 ** -21, "bf16x3": 2.0 ** -16}
ELEM_U = {"fp32": 2.0 ** -24, "fp16x3": 2.0 ** -24, "bf16x3": 2.0 ** -16, "tf32": 2.0 ** -11,
          "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,nb", [(7, 64), (200, 64), (517, 128), (1000, 256)])
def test_chol_mixed_dyadic_exact(prec, n, nb):
    A, L0 = inputs.dyadic_chol(n, seed=950 + n)
    F, info = api.chol_factor_mixed(A.to(DEV), prec=prec, nb=nb)
    assert int(info.item()) == 0
    Fd = F.to(torch.float64).cpu()
    assert torch.equal(torch.tril(Fd), L0)
    assert torch.equal(torch.triu(Fd, 1), torch.triu(L0.t(), 1))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,nb", [(300, 64), (1100, 256), (2100, 256)])
def test_chol_mixed_matches_oracle_elementwise(prec, n, nb):
    A = inputs.spd(n, seed=n).numpy()
    F, info = api.chol_factor_mixed(torch.from_numpy(A).to(DEV), prec=prec, nb=nb)
    assert int(info.item()) == 0
    Lg = np.tril(F.cpu().numpy().astype(np.float64))
    Wo, info_o = M.chol_lowprec(A, nb, prec)
    assert info_o == 0
    Lo = np.tril(Wo)
    bound = n * ELEM_U[prec] * (np.abs(Lo) @ np.abs(Lo.T)).max()
    assert np.abs(Lg - Lo).max() <= bound


# the (precision, kappa) pairs with kappa * u_p <= 10 (M^{-1} A = I + E with
# ||E|| of order one or less); the others are outside the refinement's range
CONVERGING = [(p, k) for p in PRECS for k in (1e2, 1e4, 1e6) if k * UNIT[p] <= 10.0]


@pytest.mark.parametrize("prec,kappa", CONVERGING)
def test_chol_gmresir_small(prec, kappa):
    n = 600
    A = inputs.haar_spd(n, kappa)
    b = A @ inputs.normal((n,), 6)
    x, st = api.solve_chol_mixed(A.to(DEV), b.to(DEV), prec=prec, nb=128, tol=1e-14, max_outer=30,
                                 restart_m=50)
    assert st["converged"], st
    An = np.asfortranarray(A.numpy())
    assert oracle.backward_error(An, x.cpu().numpy(), b.numpy())[0] <= 1e-14


def test_chol_gmresir_several_rhs():
    n = 700
    A = inputs.haar_spd(n, 1e4, device=DEV)
    B = A @ inputs.normal((n, 3), 6, DEV)
    X, sts = api.solve_chol_mixed(A, B, prec="fp16x3", nb=256, max_outer=20)
    An = np.asfortranarray(A.cpu().numpy())
    for j in range(3):
        assert sts[j]["converged"]
        assert oracle.backward_error(An, X[:, j].cpu().numpy(), B[:, j].cpu().numpy())[0] <= 1e-14


@pytest.mark.parametrize("n,k", [(10, 3), (300, 0), (300, 150), (700, 600)])
def test_chol_mixed_not_spd(n, k):
    A = inputs.spd(n, seed=11).numpy()
    A[k, k] = -1.0
    _, info_o = M.chol_lowprec(A, 128, "fp16x3")
    F, info = api.chol_factor_mixed(torch.from_numpy(A).to(DEV), prec="fp16x3", nb=128)
    assert info_o == k + 1
    assert int(info.item()) == k + 1
