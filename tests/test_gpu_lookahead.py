"""Look-ahead in the blocked LU (the next outer block's panels factored on a
second, high-priority stream while the rest of the trailing update runs): the
same operations on every element in the same order, so the factors, pivots
and info must be bit-for-bit those of the factorisation without it, for the
tensor-core (fp16x3, bf16), SIMT FP32 and FP64 paths, with ragged last blocks."""
import pytest
import torch

from paper_1511_07174_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _both(fn):
    old = api.get_lookahead()
    try:
        api.set_lookahead(False)
        a = fn()
        torch.cuda.synchronize()
        api.set_lookahead(True)
        b = fn()
        torch.cuda.synchronize()
    finally:
        api.set_lookahead(old)
    return a, b


@pytest.mark.parametrize("prec", ["fp16x3", "bf16", "fp32"])
@pytest.mark.parametrize("n,nb", [(1100, 128), (2100, 256), (700, 64)])
def test_mixed_lookahead_identical(prec, n, nb):
    A = inputs.uniform(n, seed=n + 3, device=DEV)
    (F0, p0, i0), (F1, p1, i1) = _both(lambda: api.lu_factor_mixed(A, prec=prec, nb=nb))
    assert int(i0.item()) == int(i1.item()) == 0
    assert torch.equal(p0, p1)
    assert torch.equal(F0, F1)


@pytest.mark.parametrize("n,nb", [(1100, 128), (2100, 256)])
def test_fp64_lookahead_identical(n, nb):
    A = inputs.uniform(n, seed=n + 5, device=DEV)
    (L0, p0, i0), (L1, p1, i1) = _both(lambda: api.lu_factor(A, nb=nb))
    assert int(i0.item()) == int(i1.item()) == 0
    assert torch.equal(p0, p1)
    assert torch.equal(L0, L1)
