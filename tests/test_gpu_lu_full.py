"""FP64 LU at the full measured size (n = 8192, 16 right-hand sides), checked on
what the oracle can compute one by one or at any size:
  * the first 64 pivots and the first 64 columns of L / rows of U against the
    oracle's first 64 elimination steps on the same matrix (the later
    interchanges move rows of L, so they are applied to the oracle's partial
    result before comparing);
  * backward error <= 1e-14 for every right-hand side (oracle FP64 matvec);
  * |l_ij| <= 1.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1511_07174_gb300 import api, inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
DEV = "cuda:0"


def test_lu_n8192_16rhs():
    n, nrhs, k = 8192, 16, 64
    A = inputs.uniform(n, seed=0)
    X_true = inputs.normal((n, nrhs), seed=1)
    B = A @ X_true
    LU, ipiv, info = api.lu_factor(A.to(DEV), nb=256)
    X = api.lu_solve(LU, ipiv, B.to(DEV))
    torch.cuda.synchronize()
    assert int(info.item()) == 0
    An = np.asfortranarray(A.numpy())
    beta = oracle.backward_error(An, X.cpu().numpy(), B.numpy())
    assert beta.max() <= 1e-14
    LUg = LU.cpu().numpy()
    ipg = ipiv.cpu().numpy()
    assert np.abs(np.tril(LUg, -1)).max() <= 1.0
    assert oracle.min_pivot_gap(An, k) > 1e-10
    W, ipo, _ = oracle.getrf(An, ksteps=k)
    assert np.array_equal(ipg[:k], ipo[:k])
    # apply the GPU's later interchanges to the oracle's partially eliminated rows
    for j in range(k, n):
        p = ipg[j] - 1
        if p != j:
            W[[j, p], :] = W[[p, j], :]
    scale = np.abs(W[:, :k]).max()
    assert np.abs(LUg[:, :k] - W[:, :k]).max() <= 1e-12 * scale
    assert np.abs(LUg[:k, :] - W[:k, :]).max() <= 1e-11 * np.abs(W[:k, :]).max()
