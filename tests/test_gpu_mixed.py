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
from oracle import gmres as G
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
    less; the test asks for it where kappa * u_p <= 10. Two more cases converge
    on the oracle with the same factors (bf16x3 at 1e6 with GMRES(50); bf16 at
    1e4 with GMRES(128) restarted 4 times per refinement step) and are asked
    for with those settings."""
    return kappa * UNIT[prec] <= 10.0 or (prec, kappa) in LONGER


LONGER = {("bf16x3", 1e6): (50, 1), ("bf16", 1e4): (128, 4)}
# kappa * u_p from 500 to 4000: the factors are too weak a preconditioner;
# restarted GMRES(128) stalls on them (the oracle stalls on the same factors)
STALL = [("bf16", 1e6), ("fp16", 1e6), ("tf32", 1e6)]


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


def _haar_system(n, kappa):
    UV = (inputs.haar(n, 4), inputs.haar(n, 5))
    A = inputs.haar_kappa(n, kappa, UV=UV)
    x_true = inputs.normal((n,), 6)
    return A, A @ x_true


# element-by-element bound of the GPU factors against the oracle's with the
# same pivots: n operations per entry, each at most one rounding apart
ELEM_U = {"fp32": 2.0 ** -24, "fp16x3": 2.0 ** -24, "bf16x3": 2.0 ** -16, "tf32": 2.0 ** -11,
          "bf16": 2.0 ** -8, "fp16": 2.0 ** -11}


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n,nb,seed", [(300, 64, 300), (1100, 256, 1100), (2100, 256, 2101)])
def test_mixed_factors_match_oracle_elementwise(prec, n, nb, seed):
    """The GPU's low-precision factors, entry by entry, against the oracle's
    low-precision LU (oracle/mixed.py) run on the same input with the GPU's
    pivot sequence forced (random inputs have near-ties that either side may
    break: over a whole n = 2100 matrix the smallest gap is ~1e-5).

    Reading of the panel precision: the GPU panel and substitutions do FP32
    arithmetic (one rounding per fused multiply-add), the oracle does each step
    in FP64 and rounds the stored value to FP32; the two are at most one FP32
    ulp apart per operation. The update products take the same rounded operands
    on both sides and differ in the order of the FP32 accumulation, and, when a
    one-ulp difference moves an operand across a rounding boundary of the
    16-bit / TF32 format, by one unit u_p of that format. An entry passes
    through at most n such operations, each at most max(|L||U|) in size, and
    partial pivoting keeps |l| <= 1, so
        |F_gpu - F_oracle| <= n * u * max(|L||U|),
    u = 2^-24 for fp32 and fp16x3 (whose split keeps the product to FP32
    accuracy), u_p of the format otherwise (bf16x3: 2^-16).
    Every GPU pivot must be a largest candidate of its column in the oracle's
    arithmetic up to that same relative margin."""
    A = inputs.uniform(n, seed=seed).numpy()
    W, ipiv, info = _mixed(torch.from_numpy(A), prec, nb)
    assert info == 0
    p = oracle.perm_from_ipiv(ipiv, n)
    assert np.array_equal(np.sort(p), np.arange(n))
    Wo, ipo, info_o, slack = M.lu_lowprec(A, nb, prec, force_ipiv=ipiv)
    assert info_o == 0
    Lo, Uo = oracle.unpack_lu(Wo)
    bound = n * ELEM_U[prec] * (np.abs(Lo) @ np.abs(Uo)).max()
    assert slack <= n * ELEM_U[prec] * (np.abs(Lo) @ np.abs(Uo)).max() / np.abs(np.diag(Uo)).min()
    assert np.abs(W - Wo).max() <= bound


# every (precision, kappa) pair except the three that stall (tested below)
CONVERGING = [(p, k) for p in PRECS for k in (1e2, 1e4, 1e6) if (p, k) not in STALL]


@pytest.mark.parametrize("prec,kappa", CONVERGING)
def test_gmresir_small(prec, kappa):
    assert _expected_to_converge(prec, kappa)
    n = 600
    A, b = _haar_system(n, kappa)
    m, cycles = LONGER.get((prec, kappa), (50, 1))
    x, st = api.solve_mixed(A.to(DEV), b.to(DEV), prec=prec, nb=128, tol=1e-14,
                            max_outer=30, restart_m=m, restarts=cycles)
    xg = x.cpu().numpy()
    An = np.asfortranarray(A.numpy())
    assert st["converged"], st
    assert oracle.backward_error(An, xg, b.numpy())[0] <= 1e-14
    LUo, ipo, _ = oracle.getrf(An)
    xo = oracle.getrs(LUo, ipo, b.numpy())[:, 0]
    assert np.abs(xg - xo).max() <= kappa * 1e-13 * np.abs(xo).max()


@pytest.mark.parametrize("prec,kappa", STALL)
def test_gmresir_stall_matches_oracle(prec, kappa):
    """Where the low-precision factors are too weak a preconditioner, the GPU
    refinement must say so (not converged, the backward error it reports is the
    one the oracle's FP64 matvec measures), and the oracle's GMRES-IR on the
    same factors, with the same GMRES(128) x 4 cycles, stalls at the same level
    (within a factor 100)."""
    n = 600
    A, b = _haar_system(n, kappa)
    F, ipiv, info = api.lu_factor_mixed(A.to(DEV), prec=prec, nb=128)
    x, st = api.gmresir(A.to(DEV), F, ipiv, b.to(DEV), tol=1e-14, max_outer=3, restart_m=128,
                        restarts=4)
    An = np.asfortranarray(A.numpy())
    beta_gpu = oracle.backward_error(An, x.cpu().numpy(), b.numpy())[0]
    assert not st["converged"]
    assert abs(st["beta"] - beta_gpu) <= 1e-3 * beta_gpu + 1e-16
    W = F.cpu().numpy().astype(np.float64)
    ap = M.apply_minv_factory(W, ipiv.cpu().numpy())
    _, sto = G.gmres_ir(A.numpy(), b.numpy(), ap, tol=1e-14, m=128, tau=1e-8, max_outer=3,
                        restarts=4)
    beta_o = sto["beta_history"][-1]
    assert not sto["converged"]
    assert beta_gpu > 1e-10 and beta_o > 1e-10
    assert 0.01 <= beta_gpu / beta_o <= 100.0, (beta_gpu, beta_o)


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



@pytest.mark.parametrize("n", [600, 2100])
def test_substitution_cap_gives_the_same_result(n):
    """The refinement's substitution is a persistent grid drawing its tasks in
    order; capping its CTAs (here below the number of tasks) changes which CTA
    runs a task, not the operations: the refined x and the iteration counts
    must be identical."""
    A, b = _haar_system(n, 1e4)
    Ad, bd = A.to(DEV), b.to(DEV)
    F, ipiv, info = api.lu_factor_mixed(Ad, prec="fp16x3", nb=128)
    x0, st0 = api.gmresir(Ad, F, ipiv, bd, tol=1e-14, max_outer=10)
    old = api.get_substitution_ctas()
    try:
        api.set_substitution_ctas(3)
        x1, st1 = api.gmresir(Ad, F, ipiv, bd, tol=1e-14, max_outer=10)
    finally:
        api.set_substitution_ctas(old)
    assert torch.equal(x0, x1)
    assert (st0["outer"], st0["inner"]) == (st1["outer"], st1["inner"])
    assert st0["converged"]
