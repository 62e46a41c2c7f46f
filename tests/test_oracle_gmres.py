"""Pins for the GMRES / GMRES-IR oracle and for the low-precision LU oracle.

* Krylov theory: with k distinct eigenvalues GMRES terminates in k steps and
  not earlier; the Arnoldi relation A V_k = V_{k+1} H_k holds with V
  orthonormal; residual norms never increase; full GMRES equals a direct solve.
* An exact preconditioner makes GMRES converge in one step.
* Rounding helpers agree with library conversions (numpy float16, torch
  bfloat16) and with hand-computed TF32 roundings.
* The low-precision LU recovers exactly representable factors bit for bit in
  every update precision, and classical theory bounds GMRES-IR's outer steps.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import gmres as G
from oracle import mixed as M
from paper_1511_07174_gb300 import inputs


def test_gmres_distinct_eigenvalues():
    n, k = 60, 5
    rng = np.random.default_rng(0)
    eig = np.repeat(np.array([1.0, 2.0, 3.5, -1.5, 7.0]), n // k)
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(eig) @ Q.T
    b = rng.standard_normal(n)
    d, steps, hist = G.gmres(lambda v: A @ v, b, m=n, tol=1e-12)
    assert steps == k
    assert hist[k - 1] > 1e-6 * np.linalg.norm(b)
    assert np.linalg.norm(A @ d - b) <= 1e-10 * np.linalg.norm(b)


def test_arnoldi_relation():
    n, k = 40, 12
    A = inputs.uniform(n, seed=11).numpy()
    v0 = np.ones(n)
    V, H = G.arnoldi(lambda v: A @ v, v0, k)
    assert np.abs(V.T @ V - np.eye(k + 1)).max() <= 1e-13
    assert np.abs(A @ V[:, :k] - V @ H).max() <= 1e-13
    assert np.abs(np.tril(H, -2)).max() == 0.0


def test_gmres_monotone_and_full():
    n = 30
    A = inputs.uniform(n, seed=12).numpy() + 2 * np.eye(n)
    b = np.sin(np.arange(n, dtype=np.float64))
    d, steps, hist = G.gmres(lambda v: A @ v, b, m=n, tol=1e-14)
    assert all(hist[i + 1] <= hist[i] * (1 + 1e-12) for i in range(len(hist) - 1))
    assert np.abs(d - np.linalg.solve(A, b)).max() <= 1e-10


def test_gmres_restart_converges():
    n = 50
    A = inputs.uniform(n, seed=13).numpy() + 8 * np.eye(n)
    b = np.ones(n)
    d, steps, hist = G.gmres(lambda v: A @ v, b, m=5, tol=1e-12, restarts=40)
    assert np.linalg.norm(A @ d - b) <= 1e-11 * np.linalg.norm(b)


def test_gmres_exact_preconditioner_one_step():
    n = 64
    A = inputs.uniform(n, seed=14).numpy()
    LU, ipiv, _ = oracle.getrf(np.asfortranarray(A))
    minv = lambda v: oracle.getrs(LU, ipiv, v)[:, 0]
    r = np.cos(np.arange(n, dtype=np.float64))
    d, steps, hist = G.gmres(lambda v: minv(A @ v), minv(r), m=20, tol=1e-10)
    assert steps == 1


def test_round_helpers_against_libraries():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 4, 10000)).astype(np.float32)
    bt = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy().astype(np.float64)
    assert np.array_equal(M.round_bf16(x), bt)
    assert np.array_equal(M.round_fp16(x), x.astype(np.float16).astype(np.float64))
    # TF32 keeps 10 explicit mantissa bits; halfway cases round away from zero
    one = np.float32(1.0)
    tests = {1.0 + 2.0 ** -11: 1.0 + 2.0 ** -10,          # tie -> away
             1.0 + 2.0 ** -12: 1.0,                       # below half -> down
             -(1.0 + 3 * 2.0 ** -11): -(1.0 + 2 * 2.0 ** -10),
             1.0 + 2.0 ** -10: 1.0 + 2.0 ** -10}
    for v, want in tests.items():
        assert M.round_tf32(np.array([v], dtype=np.float32))[0] == want
    assert one == 1.0


def test_sliver_exponent_range():
    vals = np.array([1e-20, 3e-5, 0.7, 1.0, 1234.5, 6e4, 2.0 ** 14, 2.0 ** 15 - 1])
    e = M.sliver_exponent(vals)
    s = np.ldexp(vals, e)
    assert ((s >= 2.0 ** 14) & (s < 2.0 ** 15)).all()
    assert M.sliver_exponent(np.array([0.0]))[0] == 0
    assert M.sliver_exponent(np.array([1e-35]))[0] == M.SCALE_CLAMP     # clamped


@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16", "fp16", "fp16x3", "bf16x3"])
@pytest.mark.parametrize("n,nb", [(1, 4), (37, 8), (96, 32)])
def test_lowprec_lu_dyadic_exact(prec, n, nb):
    A, L0, U0, perm = inputs.dyadic_lu(n, seed=500 + n)
    W, ipiv, info = M.lu_lowprec(A.numpy(), nb, prec)
    L, U = oracle.unpack_lu(W)
    assert info == 0
    assert np.array_equal(L, L0.numpy()) and np.array_equal(U, U0.numpy())
    assert np.array_equal(oracle.perm_from_ipiv(ipiv, n), perm.numpy())


@pytest.mark.parametrize("prec", ["tf32", "bf16", "fp16", "fp16x3", "bf16x3"])
@pytest.mark.parametrize("n,nb,ko", [(37, 8, 16), (150, 16, 64), (200, 32, 96)])
def test_lowprec_lu_two_level_dyadic_exact(prec, n, nb, ko):
    """Two-level delayed updating (super-blocks of ko columns, ragged last
    ones) reaches the same exact dyadic factors: every intermediate is a short
    dyadic rational, so any misplaced block, range or operand order shows."""
    A, L0, U0, perm = inputs.dyadic_lu(n, seed=510 + n)
    W, ipiv, info = M.lu_lowprec(A.numpy(), nb, prec, ko=ko)
    L, U = oracle.unpack_lu(W)
    assert info == 0
    assert np.array_equal(L, L0.numpy()) and np.array_equal(U, U0.numpy())
    assert np.array_equal(oracle.perm_from_ipiv(ipiv, n), perm.numpy())


@pytest.mark.parametrize("prec", ["fp32", "fp16x3", "bf16"])
def test_lowprec_lu_two_level_reduces_to_one_level(prec):
    """ko = nb is the one-level algorithm, bit for bit; a larger ko gives a
    factorisation of the same quality: ||PA - LU|| within the one-level bound,
    and the same pivots where the update is accurate enough that no near-tie
    of this input flips (fp32, fp16x3; bf16's 2^-8 rounding does flip some)."""
    n, nb = 300, 32
    A = inputs.uniform(n, seed=301).numpy()
    W1, p1, _ = M.lu_lowprec(A, nb, prec)
    W2, p2, _ = M.lu_lowprec(A, nb, prec, ko=nb)
    assert np.array_equal(W1, W2) and np.array_equal(p1, p2)
    W4, p4, _ = M.lu_lowprec(A, nb, prec, ko=4 * nb)
    if prec != "bf16":
        assert np.array_equal(p1, p4)
    u = {"fp32": 2.0 ** -24, "fp16x3": 2.0 ** -21, "bf16": 2.0 ** -8}[prec]
    L, U = oracle.unpack_lu(W4)
    pr = oracle.perm_from_ipiv(p4, n)
    assert np.abs(A[pr] - L @ U).max() <= 8 * np.sqrt(n) * u * (np.abs(L) @ np.abs(U)).max()
    with pytest.raises(ValueError):
        M.lu_lowprec(A, nb, prec, ko=nb + 1)


def test_lowprec_lu_fp32_close_to_fp64():
    n = 128
    A = inputs.uniform(n, seed=0).numpy()
    W, ipiv, info = M.lu_lowprec(A, 32, "fp32")
    LU, ipiv64, _ = oracle.getrf(np.asfortranarray(A))
    assert np.array_equal(ipiv, ipiv64)
    assert np.abs(W - LU).max() <= 1e-4 * np.abs(LU).max()


@pytest.mark.parametrize("prec,kappa,max_outer", [("fp32", 1e2, 3), ("bf16", 1e4, 10),
                                                   ("fp16", 1e4, 10), ("fp16x3", 1e6, 4)])
def test_gmres_ir_oracle_converges(prec, kappa, max_outer):
    n = 160
    A = inputs.haar_kappa(n, kappa, seed_u=4, seed_v=5).numpy()
    x_true = inputs.normal((n,), 6).numpy()
    b = A @ x_true
    W, ipiv, info = M.lu_lowprec(A, 32, prec)
    x, st = G.gmres_ir(A, b, M.apply_minv_factory(W, ipiv), tol=1e-14, m=50, tau=1e-8,
                       max_outer=max_outer)
    assert st["converged"], st
    assert oracle.backward_error(A, x, b)[0] <= 1e-14
    assert np.abs(x - x_true).max() <= 1e-14 * kappa * 100 * np.abs(x_true).max()


def test_split_product_accuracy():
    """hi*hi + hi*lo + lo*hi recovers the FP32 product to ~2^-21 (fp16x3) and
    ~2^-16 (bf16x3) relative, far better than one 16-bit pass."""
    rng = np.random.default_rng(3)
    A = rng.standard_normal((64, 48))
    B = rng.standard_normal((48, 40))
    exact = A @ B
    scale = np.abs(A).dot(np.abs(B)).max()
    err = {p: np.abs(M.lowprec_product(A, B, p) - exact).max() / scale
           for p in ("fp16", "fp16x3", "bf16", "bf16x3", "fp32")}
    assert err["fp16x3"] <= 2.0 ** -20 and err["fp16x3"] < err["fp16"] / 50
    assert err["bf16x3"] <= 2.0 ** -15 and err["bf16x3"] < err["bf16"] / 50


# ------------------------------- pivot-gap diagnostic of the low-precision LU
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16", "fp16", "fp16x3", "bf16x3"])
@pytest.mark.parametrize("a,b,gap", [(0.375, -0.5, 0.25), (0.5, -0.5, 0.0), (0.25, -0.75, 0.5)])
def test_lowprec_gap_hand_built(prec, a, b, gap):
    """The 3 x 3 matrices whose gaps are known exactly (step 0: 1/2; step 1:
    (max - min) / max of |a|, |b|, visible only after elimination). Every value
    and product here is exact in all six precisions, with nb = 1 (the update
    between the columns runs in the low precision) and nb = 3 (none)."""
    A = np.array([[2.0, 1.0, 0.0], [1.0, 0.5 + a, 0.0], [1.0, 0.5 + b, 1.0]])
    for nb in (1, 3):
        _, _, _, g = M.lu_lowprec(A, nb, prec, with_gap=True)
        assert g == gap
    # a single candidate never lowers it; an exact tie in column 0 gives 0
    assert M.lu_lowprec(np.array([[5.0]]), 1, prec, with_gap=True)[3] == 1.0
    assert M.lu_lowprec(np.array([[1.0, 2.0], [-1.0, 3.0]]), 1, prec, with_gap=True)[3] == 0.0


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp16x3"])
@pytest.mark.parametrize("n,nb", [(37, 8), (96, 32)])
def test_lowprec_forced_pivots(prec, n, nb):
    """Forced pivots: the generator's own row order on an exact dyadic product
    recovers L and U bit for bit with no shortfall; the oracle's own pivots
    reproduce its free run exactly."""
    A, L0, U0, perm = inputs.dyadic_lu(n, seed=800 + n)
    W, ipiv, info = M.lu_lowprec(A.numpy(), nb, prec)
    Wf, ipf, infof, slack = M.lu_lowprec(A.numpy(), nb, prec, force_ipiv=ipiv)
    assert np.array_equal(Wf, W) and np.array_equal(ipf, ipiv) and slack == 0.0
    # pivots that reproduce P0 without being the searched ones are impossible here
    # (|l| < 1: every pivot is the strict maximum), so forcing ipiv = the searched
    # one is the only zero-slack choice; forcing the identity is not
    _, _, _, s_id = M.lu_lowprec(A.numpy(), nb, prec, force_ipiv=np.arange(1, n + 1))
    assert (s_id > 0.0) == (not np.array_equal(ipiv, np.arange(1, n + 1)))


def test_lowprec_forced_pivot_shortfall_known():
    """Column 0 holds 0.5, -1, 0.75: forcing row 2 (|0.75|) falls short of the
    maximum |-1| by exactly 1/4; forcing row 1 by 0."""
    A = np.array([[0.5, 0.0, 0.0], [-1.0, 1.0, 0.0], [0.75, 0.0, 1.0]])
    assert M.lu_lowprec(A, 3, "fp32", force_ipiv=[3, 2, 3])[3] == 0.25
    assert M.lu_lowprec(A, 3, "fp32", force_ipiv=[2, 3, 3])[3] == 0.0


# ------------------------------------------------------------- BiCGSTAB oracle
def _nonsym(n, seed, shift):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, (n, n)) + shift * np.eye(n)


def test_bicgstab_residual_recurrence_is_true_residual():
    """The updated residual r_i must equal b - A x_i at every step (a dropped or
    mis-signed term in the x or r update breaks it)."""
    n = 80
    A = _nonsym(n, 1, 12.0)
    b = np.random.default_rng(2).normal(size=n)
    for k in range(1, 8):
        x, info = G.bicgstab(A, b, tol=0.0, max_iter=k)
        true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert abs(true - info["relres"][-1]) <= 1e-12


def test_bicgstab_multiple_of_identity_one_step():
    n = 17
    b = np.arange(1.0, n + 1)
    x, info = G.bicgstab(3.0 * np.eye(n), b, tol=1e-15, max_iter=10)
    assert info["iterations"] == 1 and info["converged"] and not info["breakdown"]
    assert np.abs(x - b / 3.0).max() <= 4 * 2.0 ** -53 * np.abs(b / 3.0).max()


def test_bicgstab_exact_preconditioner_one_step():
    n = 40
    A = _nonsym(n, 3, 2.0)
    b = np.random.default_rng(4).normal(size=n)
    Ainv = np.linalg.inv(A)
    x, info = G.bicgstab(A, b, tol=1e-12, max_iter=5, apply_minv=lambda v: Ainv @ v)
    assert info["iterations"] == 1 and info["converged"]


def test_bicgstab_converges_to_direct_solution():
    n = 120
    A = _nonsym(n, 5, 15.0)
    b = np.random.default_rng(6).normal(size=n)
    x, info = G.bicgstab(A, b, tol=1e-13, max_iter=200)
    assert info["converged"]
    xd = np.linalg.solve(A, b)
    assert np.abs(x - xd).max() <= 1e-11 * np.abs(xd).max()


def test_bicgstab_matches_scipy_iterates():
    """SciPy's independent BiCGSTAB, run for the same number of steps from the
    same start, reaches the same iterate (both FP64; rounding apart)."""
    sla = pytest.importorskip("scipy.sparse.linalg")
    n = 60
    A = _nonsym(n, 7, 10.0)
    b = np.random.default_rng(8).normal(size=n)
    for k in (1, 2, 5):
        x, _ = G.bicgstab(A, b, tol=0.0, max_iter=k)
        xs, _ = sla.bicgstab(A, b, x0=np.zeros(n), rtol=0.0, atol=0.0, maxiter=k)
        assert np.abs(x - xs).max() <= 1e-10 * np.abs(xs).max()


# ------------------------------------------------------ low-precision Cholesky
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16", "fp16", "fp16x3", "bf16x3"])
@pytest.mark.parametrize("n,nb", [(1, 4), (37, 8), (96, 32)])
def test_lowprec_chol_dyadic_exact(prec, n, nb):
    """Integer L (diagonal 1, 2, 4; entries in [-3, 3]): every operand is exact in
    every update precision and every FP32 sum is exact, so L comes back bit for
    bit, as does the solution of L L^t x = b for an integer x."""
    A, L0 = inputs.dyadic_chol(n, seed=900 + n)
    W, info = M.chol_lowprec(A.numpy(), nb, prec)
    assert info == 0
    assert np.array_equal(np.tril(W), L0.numpy())
    x = np.arange(1.0, n + 1)
    ap = M.chol_minv_factory(W)
    assert np.array_equal(ap(A.numpy() @ x), x)


@pytest.mark.parametrize("prec,u", [("fp32", 2.0 ** -24), ("bf16", 2.0 ** -8), ("fp16x3", 2.0 ** -21)])
def test_lowprec_chol_backward_error(prec, u):
    """||A - L L^t|| <= c n u_p ||L|| ||L^t|| (Cholesky backward stability with the
    update precision's unit roundoff); the FP32 variant is close to FP64 potrf."""
    n, nb = 150, 32
    A = inputs.spd(n, seed=31).numpy()
    W, info = M.chol_lowprec(A, nb, prec)
    assert info == 0
    L = np.tril(W)
    assert np.abs(A - L @ L.T).max() <= 4 * n * u * (np.abs(L) @ np.abs(L.T)).max()
    if prec == "fp32":
        Lo, _ = oracle.potrf(np.asfortranarray(A))
        assert np.abs(L - np.tril(Lo)).max() <= 8 * n * 2.0 ** -24 * np.abs(np.tril(Lo)).max()


def test_lowprec_chol_not_spd():
    A = inputs.spd(40, seed=32).numpy()
    A[17, 17] = -1.0
    _, info = M.chol_lowprec(A, 8, "bf16")
    assert info == 18


def test_chol_gmres_ir_oracle_converges():
    """SPD system of condition 1e4 (A = U diag(s) U^t, U Haar): GMRES-IR with
    the fp16x3 Cholesky factors reaches 1e-14 (oracle FP64 matvec)."""
    n = 200
    U = inputs.haar(n, 4).numpy()
    s = 1e4 ** (-np.arange(n) / (n - 1))
    A = (U * s) @ U.T
    A = (A + A.T) / 2
    b = A @ np.random.default_rng(0).normal(size=n)
    W, info = M.chol_lowprec(A, 32, "fp16x3")
    assert info == 0
    x, st = G.gmres_ir(A, b, M.chol_minv_factory(W), tol=1e-14, m=50, max_outer=10)
    assert st["converged"]
    assert oracle.backward_error(np.asfortranarray(A), x, b)[0] <= 1e-14
