"""GPU parity of the mixed-precision path: low-precision blocked LU (tcgen05
trailing update for TF32 / BF16 / FP16, SIMT FP32) and GMRES-based refinement.

What is unique is compared exactly; the rest is checked for validity:
  * exact dyadic products L U: every precision recovers P, L and U bit for bit
    (operands of every update are exactly representable, FP32 sums are exact);
  * random inputs: the FP32 factors satisfy ||P A - L U||_max <= c u_p ||L| |U||
    with u_p the update precision's unit roundoff (c = 8 sqrt(n) for the
    rounding of both operands plus FP32 accumulation); pivots form a
    permutation and |l_ij| <= 1;
  * the tensor-core factors agree with the oracle's low-precision LU
    (oracle/mixed.py) on the same input to within that same bound;
  * GMRES-IR: backward error (oracle FP64 matvec) <= 1e-14, and the solution
    agrees with the oracle's FP64 direct solution to kappa * 1e-13.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle import mixed as M
from paper_1511_07174_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
UNIT = {"fp32": 2.0 ** -24, "tf32": 2.0 ** -11, "bf16": 2.0 ** -8, "fp16": 2.0 ** -11,
        "fp16x3": 2.0 ** -21, "bf16x3": 2.0 ** -16}
PRECS = ["fp32", "tf32", "bf16", "fp16", "fp16x3", "bf16x3"]


def _expected_to_converge(prec, kappa):
    """GMRES-IR with restarted GMRES(50) is expected to reach 1e-14 when the
    preconditioned matrix M^{-1} A = I + E has ||E|| ~ kappa u_p of order one or
    less; the test asks for it where kappa * u_p <= 10."""
    return kappa * UNIT[prec] <= 10.0


def _mixed(A, prec, nb):
    F, ipiv, info = api.lu_factor_mixed(A.to(DEV), prec=prec, nb=nb)
    torch.cuda.synchronize()
    return F.cpu().numpy().astype(np.float64), ipiv.cpu().numpy(), int(info.item())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,nb", [(7, 32), (200, 64), (517, 128), (1000, 256)])
def test_mixed_dyadic_exact(prec, n, nb):
    A, L0, U0, perm = inputs.dyadic_lu(n, seed=600 + n)
    W, ipiv, info = _mixed(A, prec, nb)
    L, U = oracle.unpack_lu(W)
    assert info == 0
    assert np.array_equal(L, L0.numpy()), np.abs(L - L0.numpy()).max()
    assert np.array_equal(U, U0.numpy()), np.abs(U - U0.numpy()).max()
    assert np.array_equal(oracle.perm_from_ipiv(ipiv, n), perm.numpy())


@pytest.mark.parametrize("prec", ["fp32", "fp16x3", "bf16"])
def test_mixed_dyadic_exact_tall_panels(prec):
    """n = 8448: the first panels (more than 8192 rows) hold two rows per
    thread in the cluster panel kernel, the later ones one; factors and
    pivots must still be exact."""
    n = 8448
    A, L0, U0, perm = inputs.dyadic_lu(n, seed=611, device=DEV)
    F, ipiv, info = api.lu_factor_mixed(A, prec=prec, nb=256)
    assert int(info.item()) == 0
    Fd = F.to(torch.float64)
    eye = torch.eye(n, dtype=torch.float64, device=DEV)
    assert torch.equal(torch.tril(Fd, -1) + eye, L0)
    assert torch.equal(torch.triu(Fd), U0)
    assert np.array_equal(oracle.perm_from_ipiv(ipiv.cpu().numpy(), n), perm.numpy())


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,nb", [(300, 64), (1100, 256)])
def test_mixed_factor_bound_and_oracle(prec, n, nb):
    A = inputs.uniform(n, seed=n).numpy()
    W, ipiv, info = _mixed(torch.from_numpy(A), prec, nb)
    assert info == 0
    p = oracle.perm_from_ipiv(ipiv, n)
    assert np.array_equal(np.sort(p), np.arange(n))
    L, U = oracle.unpack_lu(W)
    assert np.abs(np.tril(W, -1)).max() <= 1.0
    bound = 8 * math.sqrt(n) * UNIT[prec] * (np.abs(L) @ np.abs(U)).max()
    assert np.abs(A[p] - L @ U).max() <= bound
    # the oracle's low-precision LU on the same input: same bound on its factors
    Wo, ipo, _ = M.lu_lowprec(A, nb, prec)
    Lo, Uo = oracle.unpack_lu(Wo)
    po = oracle.perm_from_ipiv(ipo, n)
    assert np.abs(A[po] - Lo @ Uo).max() <= bound


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("kappa", [1e2, 1e4, 1e6])
def test_gmresir_small(prec, kappa):
    if not _expected_to_converge(prec, kappa):
        pytest.skip("kappa * u_p > 10: outside the refinement's convergence range")
    n = 600
    UV = (inputs.haar(n, 4), inputs.haar(n, 5))
    A = inputs.haar_kappa(n, kappa, UV=UV)
    x_true = inputs.normal((n,), 6)
    b = A @ x_true
    x, st = api.solve_mixed(A.to(DEV), b.to(DEV), prec=prec, nb=128, tol=1e-14,
                            max_outer=30, restart_m=50)
    xg = x.cpu().numpy()
    An = np.asfortranarray(A.numpy())
    assert st["converged"], st
    assert oracle.backward_error(An, xg, b.numpy())[0] <= 1e-14
    LUo, ipo, _ = oracle.getrf(An)
    xo = oracle.getrs(LUo, ipo, b.numpy())[:, 0]
    assert np.abs(xg - xo).max() <= kappa * 1e-13 * np.abs(xo).max()


def test_solve_mixed_several_rhs():
    """One factorisation, three right-hand sides refined one by one: each column
    reaches backward error <= 1e-14 (oracle FP64 matvec)."""
    n = 600
    A = inputs.haar_kappa(n, 1e2, device=DEV)
    X0 = inputs.normal((n, 3), 6, DEV)
    B = A @ X0
    X, sts = api.solve_mixed(A, B, prec="fp16x3", nb=128, max_outer=20)
    assert X.shape == (n, 3) and len(sts) == 3
    An = np.asfortranarray(A.cpu().numpy())
    for j in range(3):
        assert sts[j]["converged"]
        assert oracle.backward_error(An, X[:, j].cpu().numpy(), B[:, j].cpu().numpy())[0] <= 1e-14

