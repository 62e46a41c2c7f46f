"""Seeded synthetic inputs shared by the tests, the oracle comparisons and the benchmark.

This module draws random matrices and right-hand sides only; it holds none of
the solver's arithmetic. Every generator uses torch.Generator(...).manual_seed
(CPU generator unless a CUDA device is requested), returns float64 tensors and
states its recipe in its docstring. Matrices are returned as (n, n) tensors in
the usual index order A[i, j]; `colmajor` gives the column-major storage the
solver library takes.

Workloads (the paper's problem A x = b, section 2, at the sizes the solver is
measured on):
  uniform        A iid U[-1, 1]
  spd            A = B B^t / n + I, B iid N(0, 1)
  haar_kappa     A = U diag(s) V^t, U, V Haar orthogonal (QR of Gaussian,
                 sign-fixed), s_i = kappa^(-i/(n-1)) geometric from 1 to 1/kappa
  haar_spd       A = U diag(s) U^t, the SPD counterpart (same U and s)
  spd_fp32_product  B B^t / n + I with the product formed in FP32 (large n)
  batched        4096 systems, n_i iid uniform integers in [16, 256],
                 A_i iid U[-1, 1] + n_i I, nrhs_i uniform in {1..4}
  autograd       A iid U[-1, 1] + sqrt(n) I, x_true N(0, 1), g N(0, 1)
  dyadic_lu      A = P0^t L U with L unit lower in {0, +-1/4, +-1/2}, U upper,
                 integer off-diagonal in [-8, 8], diagonal in {+-1, +-2, +-4}:
                 every intermediate of the elimination is a short dyadic number
  dyadic_chol    A = L L^t, L lower, diagonal in {1, 2, 4}, off-diagonal
                 integers in [-3, 3]
"""
import math

import torch


def _gen(seed, device="cpu"):
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def colmajor(A):
    """Tensor with the same (i, j) indexing whose storage is column-major (stride (1, n))."""
    return A.t().contiguous().t()


def uniform(n, seed, device="cpu"):
    g = _gen(seed, device)
    return torch.rand((n, n), generator=g, dtype=torch.float64, device=device) * 2.0 - 1.0


def normal(shape, seed, device="cpu"):
    g = _gen(seed, device)
    return torch.randn(shape, generator=g, dtype=torch.float64, device=device)


def spd(n, seed, device="cpu"):
    B = normal((n, n), seed, device)
    return B @ B.t() / n + torch.eye(n, dtype=torch.float64, device=device)


def haar(n, seed, device="cpu"):
    """Haar-distributed orthogonal matrix: Q of the QR of an N(0,1) matrix with diag(R) > 0."""
    G = normal((n, n), seed, device)
    Q, R = torch.linalg.qr(G)
    d = torch.sign(torch.diagonal(R))
    d[d == 0] = 1.0
    return Q * d.unsqueeze(0)


def kappa_spectrum(n, kappa, device="cpu"):
    if n == 1:
        return torch.ones(1, dtype=torch.float64, device=device)
    i = torch.arange(n, dtype=torch.float64, device=device)
    return torch.pow(torch.tensor(float(kappa), dtype=torch.float64, device=device), -i / (n - 1))


def haar_kappa(n, kappa, seed_u=4, seed_v=5, device="cpu", UV=None):
    """A = U diag(s) V^t with prescribed 2-norm condition number kappa."""
    U, V = UV if UV is not None else (haar(n, seed_u, device), haar(n, seed_v, device))
    s = kappa_spectrum(n, kappa, device)
    return (U * s.unsqueeze(0)) @ V.t()


def haar_spd(n, kappa, seed_u=4, device="cpu", U=None):
    """Symmetric positive definite A = U diag(s) U^t (U Haar, s geometric from 1
    to 1/kappa), symmetrised exactly: 2-norm condition number kappa."""
    U = haar(n, seed_u, device) if U is None else U
    s = kappa_spectrum(n, kappa, device)
    A = (U * s.unsqueeze(0)) @ U.t()
    return (A + A.t()) * 0.5


def spd_fp32_product(n, seed, device="cpu"):
    """A = B B^t / n + I with B iid N(0, 1), the product formed in FP32 (fast at
    large n) and symmetrised in FP64; SPD with eigenvalues in about [1, 5]."""
    g = _gen(seed, device)
    B = torch.randn((n, n), generator=g, dtype=torch.float32, device=device)
    P = (B @ B.t()).to(torch.float64) / n
    del B
    P = (P + P.t()) * 0.5
    P.diagonal().add_(1.0)
    return P


def rhs_from_solution(A, x_true):
    return A @ x_true


def dyadic_lu(n, seed, device="cpu"):
    """(A, L, U, perm) with A = P0^t L U, where (P0^t M)[perm[i]] = M[i].
    The entries are drawn on the CPU; the product (exact in FP64 in any
    summation order: every partial sum is a multiple of 1/4 below 2^40) is
    formed on `device`."""
    g = _gen(seed)
    lvals = torch.tensor([0.0, 0.25, -0.25, 0.5, -0.5], dtype=torch.float64)
    L = lvals[torch.randint(0, 5, (n, n), generator=g)]
    L = torch.tril(L, -1) + torch.eye(n, dtype=torch.float64)
    U = torch.randint(-8, 9, (n, n), generator=g).to(torch.float64)
    dvals = torch.tensor([1.0, -1.0, 2.0, -2.0, 4.0, -4.0], dtype=torch.float64)
    U = torch.triu(U, 1) + torch.diag(dvals[torch.randint(0, 6, (n,), generator=g)])
    perm = torch.randperm(n, generator=g)
    L, U = L.to(device), U.to(device)
    M = L @ U
    A = torch.empty_like(M)
    A[perm.to(device)] = M
    return A, L, U, perm


def dyadic_chol(n, seed):
    """(A, L) with A = L L^t exactly representable."""
    g = _gen(seed)
    L = torch.randint(-3, 4, (n, n), generator=g).to(torch.float64)
    dvals = torch.tensor([1.0, 2.0, 4.0], dtype=torch.float64)
    L = torch.tril(L, -1) + torch.diag(dvals[torch.randint(0, 3, (n,), generator=g)])
    return L @ L.t(), L


def batched(batch, seed, nmin=16, nmax=256, dtype=torch.float64):
    """Uneven batch: sizes, matrices (list), right-hand sides (list), solutions (list)."""
    g = _gen(seed)
    sizes = torch.randint(nmin, nmax + 1, (batch,), generator=g).tolist()
    nrhs = torch.randint(1, 5, (batch,), generator=g).tolist()
    As, Bs, Xs = [], [], []
    for n, k in zip(sizes, nrhs):
        A = torch.rand((n, n), generator=g, dtype=torch.float64) * 2.0 - 1.0
        A += n * torch.eye(n, dtype=torch.float64)
        X = torch.randn((n, k), generator=g, dtype=torch.float64)
        As.append(A.to(dtype))
        Xs.append(X.to(dtype))
        Bs.append((A @ X).to(dtype))
    return sizes, nrhs, As, Bs, Xs


def autograd_problem(n, nrhs, seed_a=8, seed_x=10, seed_g=9, device="cpu"):
    A = uniform(n, seed_a, device) + math.sqrt(n) * torch.eye(n, dtype=torch.float64, device=device)
    x_true = normal((n, nrhs), seed_x, device)
    b = A @ x_true
    g = normal((n, nrhs), seed_g, device)
    return A, b, g
