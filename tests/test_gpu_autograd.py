"""Differentiable solve: gb = A^{-t} g through the stored factors and
gA = -gb x^t (rank-k kernel), checked against
  * the closed form at A = I (x = b, gb = g, gA = -g b^t);
  * central finite differences at n = 64, h = 1e-6, along 8 random
    directions E: |FD - <gA, E>| <= 1e-6 * max(1, |<gA, E>|) (FD truncation
    error ~h^2 ||d^3f||, rounding ~u ||f|| / h ~ 1e-10);
  * the oracle gradient (which factors A^t on its own) at n = 1024 and at
    the full n = 4096 with 8 right-hand sides: relative error <= 1e-10.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_07174_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _grads(A, b, g, method="lu"):
    A = A.to(DEV).clone().requires_grad_(True)
    b = b.to(DEV).clone().requires_grad_(True)
    x = api.solve(A, b, method)
    (x * g.to(DEV)).sum().backward()
    torch.cuda.synchronize()
    return x.detach().cpu().numpy(), A.grad.cpu().numpy(), b.grad.cpu().numpy()


@pytest.mark.parametrize("method", ["lu", "chol"])
def test_identity_closed_form(method):
    n, k = 40, 3
    A = torch.eye(n, dtype=torch.float64)
    b = inputs.normal((n, k), 1)
    g = inputs.normal((n, k), 2)
    x, gA, gb = _grads(A, b, g, method)
    assert np.allclose(x, b.numpy(), rtol=0, atol=1e-15)
    assert np.allclose(gb, g.numpy(), rtol=0, atol=1e-15)
    assert np.allclose(gA, -(g.numpy() @ b.numpy().T), rtol=1e-15, atol=1e-14)


@pytest.mark.parametrize("method", ["lu", "chol"])
def test_central_differences_n64(method):
    n, k, h = 64, 8, 1e-6
    if method == "lu":
        A = inputs.uniform(n, seed=8) + np.sqrt(n) * torch.eye(n, dtype=torch.float64)
    else:
        A = inputs.spd(n, seed=8)
    b = inputs.normal((n, k), 10)
    g = inputs.normal((n, k), 9)
    x, gA, gb = _grads(A, b, g, method)
    Ad, bd, gd = A.to(DEV), b.to(DEV), g.to(DEV)

    def f(Am):
        with torch.no_grad():
            return float((api.solve(Am, bd, "lu") * gd).sum().item())

    gen = torch.Generator().manual_seed(5)
    for _ in range(8):
        E = torch.randn((n, n), generator=gen, dtype=torch.float64).to(DEV)
        if method == "chol":   # stay SPD: symmetric direction, LU solve of the perturbed matrix
            E = (E + E.t()) / 2
        fd = (f(Ad + h * E) - f(Ad - h * E)) / (2 * h)
        ana = float((torch.from_numpy(gA).to(DEV) * E).sum().item())
        assert abs(fd - ana) <= 1e-6 * max(1.0, abs(ana)), (fd, ana)


@pytest.mark.parametrize("n,k", [(1024, 8), pytest.param(4096, 8, marks=pytest.mark.slow)])
def test_oracle_gradient(n, k):
    A, b, g = inputs.autograd_problem(n, k)
    x, gA, gb = _grads(A, b, g, "lu")
    gAo, gbo = oracle.solve_grad(np.asfortranarray(A.numpy()), x, g.numpy())
    assert np.abs(gb - gbo).max() <= 1e-10 * np.abs(gbo).max()
    assert np.abs(gA - gAo).max() <= 1e-10 * np.abs(gAo).max()


def test_rank_k_update_matches_definition():
    m, n, k = 300, 170, 21
    U = inputs.normal((m, k), 1)
    V = inputs.normal((n, k), 2)
    C0 = inputs.normal((m, n), 3)
    C = api.rank_k_update(U.to(DEV), V.to(DEV), alpha=-0.5, beta=2.0,
                          C=api.colmajor(C0.to(DEV), copy=True))
    ref = -0.5 * (U.numpy() @ V.numpy().T) + 2.0 * C0.numpy()
    assert np.abs(C.cpu().numpy() - ref).max() <= 1e-13 * np.abs(ref).max()
