"""Pins for the CPU oracle: it is checked against things other than itself.

* hand-worked fixtures (tests/golden) -- exact fractions from the definitions;
* exact integer / dyadic products L U and L L^t, which the elimination must
  recover bit for bit (every intermediate is a short dyadic number);
* Cramer's rule in exact rationals for n <= 4;
* invariants: P A = L U within the GEPP rounding bound, |l_ij| <= 1;
* special cases with known answers (identity, permutation, singular, non-SPD);
* CPU LAPACK (torch.linalg) as an independent cross-check of pivots and factors.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_1511_07174_gb300 import inputs
from tests.golden.reader import load

U64 = 2.0 ** -53


def _np(t):
    return np.asfortranarray(t.numpy())


# ----------------------------------------------------------------- golden files
def test_golden_gepp_4x4():
    g = load("gepp_4x4.txt")
    A = np.array(g["A"], dtype=np.float64)
    LU, ipiv, info = oracle.getrf(A)
    assert info == 0
    assert list(ipiv) == [int(v) for v in g["ipiv"]]
    L, U = oracle.unpack_lu(LU)
    Lx = np.array([[float(v) for v in r] for r in g["L"]])
    Ux = np.array([[float(v) for v in r] for r in g["U"]])
    assert np.abs(L - Lx).max() <= 4 * U64 * 1.0
    assert np.abs(U - Ux).max() <= 4 * U64 * 17.0
    x = oracle.getrs(LU, ipiv, np.array([float(v) for v in g["b"]]))
    assert np.abs(x[:, 0] - 1.0).max() <= 64 * U64


def test_golden_chol_3x3():
    g = load("chol_3x3.txt")
    A = np.array(g["A"], dtype=np.float64)
    L, info = oracle.potrf(A)
    assert info == 0
    Lx = np.array([[float(v) for v in r] for r in g["L"]])
    assert np.array_equal(np.tril(L), Lx)
    assert np.array_equal(np.triu(L, 1), np.triu(A, 1))   # upper untouched


# ----------------------------------------------------------- exact recoveries
@pytest.mark.parametrize("n", [1, 2, 3, 7, 16, 33, 64, 150])
def test_dyadic_lu_exact(n):
    A, L0, U0, perm = inputs.dyadic_lu(n, seed=100 + n)
    LU, ipiv, info = oracle.getrf(_np(A))
    assert info == 0
    L, U = oracle.unpack_lu(LU)
    assert np.array_equal(L, L0.numpy())
    assert np.array_equal(U, U0.numpy())
    assert np.array_equal(oracle.perm_from_ipiv(ipiv, n), perm.numpy())


@pytest.mark.parametrize("n", [1, 2, 5, 31, 64, 100])
def test_dyadic_chol_exact(n):
    A, L0 = inputs.dyadic_chol(n, seed=200 + n)
    An = _np(A)
    L, info = oracle.potrf(An)
    assert info == 0
    assert np.array_equal(np.tril(L), L0.numpy())
    assert np.array_equal(np.triu(L, 1), np.triu(An, 1))


@pytest.mark.parametrize("n", [1, 5, 40, 120])
def test_dyadic_substitution_exact(n):
    A, L0, U0, perm = inputs.dyadic_lu(n, seed=300 + n)
    g = torch.Generator().manual_seed(n)
    X = torch.randint(-4, 5, (n, 3), generator=g).to(torch.float64)
    B = A @ X
    LU, ipiv, info = oracle.getrf(_np(A))
    Xs = oracle.getrs(LU, ipiv, B.numpy())
    assert np.array_equal(Xs, X.numpy())
    Ac, Lc = inputs.dyadic_chol(n, seed=400 + n)
    Bc = Ac @ X
    Lf, info = oracle.potrf(_np(Ac))
    assert np.array_equal(oracle.potrs(Lf, Bc.numpy()), X.numpy())


# ------------------------------------------------------------------- Cramer
def _det(M):
    n = len(M)
    total = Fraction(0)
    for p in itertools.permutations(range(n)):
        inv = sum(1 for a in range(n) for b in range(a + 1, n) if p[a] > p[b])
        term = Fraction(1)
        for i in range(n):
            term *= M[i][p[i]]
        total += -term if inv % 2 else term
    return total


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("seed", range(6))
def test_cramer(n, seed):
    g = torch.Generator().manual_seed(1000 * n + seed)
    while True:
        Ai = torch.randint(-9, 10, (n, n), generator=g)
        M = [[Fraction(int(v)) for v in row] for row in Ai.tolist()]
        D = _det(M)
        if D != 0:
            break
    b = [Fraction(int(v)) for v in torch.randint(-9, 10, (n,), generator=g).tolist()]
    x_exact = []
    for k in range(n):
        Mk = [row[:] for row in M]
        for i in range(n):
            Mk[i][k] = b[i]
        x_exact.append(_det(Mk) / D)
    # exact inverse for the condition number
    inv = [[None] * n for _ in range(n)]
    for j in range(n):
        e = [Fraction(int(i == j)) for i in range(n)]
        for k in range(n):
            Mk = [row[:] for row in M]
            for i in range(n):
                Mk[i][k] = e[i]
            inv[k][j] = _det(Mk) / D
    anorm = max(sum(abs(v) for v in row) for row in M)
    ainv = max(sum(abs(v) for v in row) for row in inv)
    kappa = float(anorm * ainv)
    A = np.array([[float(v) for v in row] for row in M])
    LU, ipiv, info = oracle.getrf(A)
    assert info == 0
    x = oracle.getrs(LU, ipiv, np.array([float(v) for v in b]))[:, 0]
    xe = np.array([float(v) for v in x_exact])
    err = np.abs(x - xe).max() / max(np.abs(xe).max(), 1e-300)
    assert err <= 4 * n * U64 * kappa + 4 * U64


# ----------------------------------------------------------------- invariants
@pytest.mark.parametrize("n", [50, 200])
def test_gepp_invariants(n):
    A = _np(inputs.uniform(n, seed=n))
    LU, ipiv, info = oracle.getrf(A)
    assert info == 0
    L, U = oracle.unpack_lu(LU)
    p = oracle.perm_from_ipiv(ipiv, n)
    R = A[p] - L @ U
    gamma = 3 * n * U64 / (1 - 3 * n * U64)
    bound = gamma * np.abs(np.abs(L) @ np.abs(U)).sum(axis=1).max()
    assert np.abs(R).sum(axis=1).max() <= bound
    assert np.abs(np.tril(LU, -1)).max() <= 1.0


@pytest.mark.parametrize("n", [50, 200])
def test_chol_invariants(n):
    A = _np(inputs.spd(n, seed=n))
    L, info = oracle.potrf(A)
    assert info == 0
    Lt = np.tril(L)
    assert (np.diag(Lt) > 0).all()
    R = A - Lt @ Lt.T
    assert np.abs(R).max() <= 4 * (n + 1) * U64 * np.abs(Lt @ Lt.T).max() * 4


# -------------------------------------------------------------- special cases
def test_identity_and_diagonal():
    n = 9
    LU, ipiv, info = oracle.getrf(np.eye(n))
    assert info == 0 and list(ipiv) == list(range(1, n + 1))
    assert np.array_equal(LU, np.eye(n))
    d = np.diag(np.arange(1.0, n + 1))
    LU, ipiv, info = oracle.getrf(d)
    assert list(ipiv) == list(range(1, n + 1)) and np.array_equal(LU, d)


def test_permutation_matrix():
    n = 8
    perm = np.array([3, 0, 7, 5, 1, 2, 6, 4])
    P = np.eye(n)[perm]
    LU, ipiv, info = oracle.getrf(P)
    assert info == 0
    assert np.array_equal(LU, np.eye(n))
    p = oracle.perm_from_ipiv(ipiv, n)
    assert np.array_equal(P[p], np.eye(n))


def test_upper_dominant_no_pivoting():
    n = 12
    A = np.triu(np.ones((n, n))) + np.diag(np.full(n, 10.0))
    LU, ipiv, info = oracle.getrf(A)
    assert list(ipiv) == list(range(1, n + 1))
    assert np.array_equal(LU, A)


def test_singular_zero_column():
    n, k = 10, 4
    A = _np(inputs.uniform(n, seed=7))
    A[:, k] = 0.0
    LU, ipiv, info = oracle.getrf(A)
    assert info == k + 1
    assert ipiv[k] == k + 1          # idamax of an all-zero column picks the first row


def test_not_spd():
    n, k = 6, 3
    A = np.eye(n) * 2.0
    A[k, k] = -1.0
    L, info = oracle.potrf(A)
    assert info == k + 1


def test_n_one_and_empty():
    LU, ipiv, info = oracle.getrf(np.array([[-3.0]]))
    assert info == 0 and list(ipiv) == [1] and LU[0, 0] == -3.0
    LU, ipiv, info = oracle.getrf(np.zeros((0, 0)))
    assert info == 0 and len(ipiv) == 0


# ------------------------------------------------------------ LAPACK crosscheck
@pytest.mark.parametrize("n", [10, 100, 512])
def test_lapack_crosscheck(n):
    A = inputs.uniform(n, seed=0 if n == 512 else n)
    LUl, pivl = torch.linalg.lu_factor(A)
    LU, ipiv, info = oracle.getrf(_np(A))
    assert oracle.min_pivot_gap(_np(A)) > 1e-10
    assert np.array_equal(ipiv, pivl.numpy().astype(np.int32))
    assert np.abs(LU - LUl.numpy()).max() <= 1e-11 * max(1.0, np.abs(LU).max())
    S = inputs.spd(n, seed=n)
    L, info = oracle.potrf(_np(S))
    Ll = torch.linalg.cholesky(S).numpy()
    assert np.abs(np.tril(L) - Ll).max() <= 1e-12 * np.abs(Ll).max()


# ------------------------------------------------------------ backward error
def test_backward_error_closed_form():
    A = np.array([[2.0, 0.0], [0.0, 1.0]])
    x = np.array([1.0, 1.0])
    b = np.array([2.0, 1.5])
    # r = (0, 0.5); ||A||_inf = 2; ||x||_inf = 1
    assert oracle.backward_error(A, x, b)[0] == 0.25


def test_backward_error_gepp_small():
    n = 512
    A = _np(inputs.uniform(n, seed=0))
    x_true = np.ones((n, 1))
    b = A @ x_true
    LU, ipiv, info = oracle.getrf(A)
    x = oracle.getrs(LU, ipiv, b)
    assert oracle.backward_error(A, x, b)[0] <= 1e-14


# ----------------------------------------------------------------- gradient
def test_grad_identity_closed_form():
    n, k = 5, 2
    g = np.arange(1.0, n * k + 1).reshape(n, k)
    b = np.linspace(-1, 1, n * k).reshape(n, k)
    gA, gB = oracle.solve_grad(np.eye(n), b, g)
    assert np.array_equal(gB, g)
    assert np.allclose(gA, -g @ b.T, rtol=4e-16, atol=1e-15)


def test_grad_2x2_closed_form():
    A = np.array([[3.0, 1.0], [2.0, 4.0]])
    det = 10.0
    Ainv = np.array([[4.0, -1.0], [-2.0, 3.0]]) / det
    b = np.array([[1.0], [-2.0]])
    x = Ainv @ b
    g = np.array([[0.5], [1.5]])
    gA, gB = oracle.solve_grad(A, x, g)
    assert np.allclose(gB, Ainv.T @ g, rtol=4e-16, atol=1e-15)
    assert np.allclose(gA, -(Ainv.T @ g) @ x.T, rtol=4e-16, atol=1e-15)


def test_grad_central_differences():
    n, k = 6, 2
    A = _np(inputs.uniform(n, seed=3)) + 3 * np.eye(n)
    b = np.asfortranarray(np.arange(n * k, dtype=np.float64).reshape(n, k) / 7.0)
    g = np.asfortranarray(np.cos(np.arange(n * k, dtype=np.float64)).reshape(n, k))

    def f(Am):
        LU, ipiv, _ = oracle.getrf(Am)
        return float((oracle.getrs(LU, ipiv, b) * g).sum())

    LU, ipiv, _ = oracle.getrf(A)
    x = oracle.getrs(LU, ipiv, b)
    gA, _ = oracle.solve_grad(A, x, g)
    h = 1e-6
    for (i, j) in [(0, 0), (2, 5), (5, 1), (3, 3)]:
        Ap = A.copy(order="F"); Ap[i, j] += h
        Am = A.copy(order="F"); Am[i, j] -= h
        fd = (f(Ap) - f(Am)) / (2 * h)
        assert abs(fd - gA[i, j]) <= 1e-6 * max(1.0, abs(gA[i, j]))


# ------------------------------------------------- pivot-gap diagnostic (C11)
# The diagnostic decides whether pivot vectors are compared at all, so it is
# pinned on hand-built matrices whose gaps are known exactly (dyadic entries:
# every step below is exact in FP64).
def test_min_pivot_gap_known_column():
    # column 0: |-1| wins over |0.75| -> gap (1 - 0.75) / 1 = 1/4; the 2 x 2
    # remainder has an obvious winner chosen so that its gap is larger
    A = np.array([[0.5, 0.0, 0.0], [-1.0, 1.0, 0.0], [0.75, 0.0, 1.0]], order="F")
    # after step 0 (rows 0 and 1 swapped, l = (-0.5, -0.75)): column 1 rows 1, 2
    # hold 0 + 0.5 * 1 = 0.5 and 0 + 0.75 * 1 = 0.75 -> gap (0.75 - 0.5) / 0.75 = 1/3
    assert oracle.min_pivot_gap(A) == 0.25


def test_min_pivot_gap_exact_tie():
    A = np.array([[1.0, 2.0], [-1.0, 3.0]], order="F")
    assert oracle.min_pivot_gap(A) == 0.0


def test_min_pivot_gap_single_candidate():
    assert oracle.min_pivot_gap(np.array([[3.0]], order="F")) == 1.0
    # the last column always has one candidate and never lowers the gap
    A = np.array([[4.0, 1.0], [1.0, 5.0]], order="F")
    assert oracle.min_pivot_gap(A) == 0.75
    assert oracle.min_pivot_gap(np.zeros((0, 0), order="F")) == 1.0


@pytest.mark.parametrize("a,b,gap", [(0.375, -0.5, 0.25), (0.5, -0.5, 0.0), (0.25, -0.75, 0.5)])
def test_min_pivot_gap_after_elimination(a, b, gap):
    """Column 1 before elimination holds 1, 0.5 + a, 0.5 + b (no tie among rows
    1 and 2 when a = 0.5, b = -0.5: 1.0 and 0.0); after step 0 (pivot 2, gap
    1/2, multipliers 1/2) rows 1 and 2 of column 1 hold a and b, so the gap of
    step 1 is (max - min) / max of |a|, |b|. The diagnostic must see the
    eliminated values, not the raw ones."""
    A = np.array([[2.0, 1.0, 0.0], [1.0, 0.5 + a, 0.0], [1.0, 0.5 + b, 1.0]], order="F")
    assert oracle.min_pivot_gap(A) == gap
    # only the steps asked for count: step 0 alone has gap 1/2
    assert oracle.min_pivot_gap(A, 1) == 0.5


# ---------------------------------------- k elimination steps (ksteps < n)
@pytest.mark.parametrize("n,k", [(33, 1), (33, 3), (33, 16), (64, 63)])
def test_getrf_steps_block_identity(n, k):
    """After k steps of GEPP on A, with P the first k interchanges, the array
    holds L11\\U11, U12, the multipliers L21 and the Schur complement S such
    that P A = [L11 0; L21 I] [U11 U12; 0 S]. Dyadic inputs: every product and
    sum below is exact, so the identity holds bit for bit; the first k pivots
    are those of the full factorisation and of LAPACK."""
    A, _, _, _ = inputs.dyadic_lu(n, seed=700 + n + k)
    An = _np(A)
    W, ipiv, info = oracle.getrf(An, ksteps=k)
    assert info == 0
    P = np.arange(n)
    for j in range(k):
        p = ipiv[j] - 1
        P[j], P[p] = P[p], P[j]
    B = An[P]
    L11 = np.tril(W[:k, :k], -1) + np.eye(k)
    U11 = np.triu(W[:k, :k])
    U12 = W[:k, k:]
    L21 = W[k:, :k]
    S = W[k:, k:]
    assert np.array_equal(L11 @ U11, B[:k, :k])
    assert np.array_equal(L11 @ U12, B[:k, k:])
    assert np.array_equal(L21 @ U11, B[k:, :k])
    assert np.array_equal(L21 @ U12 + S, B[k:, k:])
    _, ipiv_full, _ = oracle.getrf(An)
    assert np.array_equal(ipiv[:k], ipiv_full[:k])
    _, piv_lapack = torch.linalg.lu_factor(A)
    assert np.array_equal(ipiv[:k], piv_lapack.numpy()[:k])


def test_getrf_steps_schur_complement_random():
    """Random input: the trailing block after k steps is the Schur complement
    B22 - B21 B11^{-1} B12 of the permuted matrix (numpy solve as the library
    step), to within the rounding of k elimination steps."""
    n, k = 120, 40
    An = _np(inputs.uniform(n, seed=77))
    W, ipiv, _ = oracle.getrf(An, ksteps=k)
    P = np.arange(n)
    for j in range(k):
        p = ipiv[j] - 1
        P[j], P[p] = P[p], P[j]
    B = An[P]
    S = B[k:, k:] - B[k:, :k] @ np.linalg.solve(B[:k, :k], B[:k, k:])
    assert np.abs(W[k:, k:] - S).max() <= 1e-12 * max(1.0, np.abs(S).max())
