"""Python entry points over the C ABI (include/gbla.h).

Each function takes CUDA tensors, passes their device pointers, sizes and the
current torch stream to the matching gbla_* call, and returns tensors. Matrices
use the usual A[i, j] indexing; storage handed to the library is column-major
(stride (1, n)). Workspaces are torch allocations on the same stream.
"""
import ctypes

import torch

from . import _lib

PREC = _lib.GBLA_PREC


class GblaError(RuntimeError):
    def __init__(self, name, rc):
        self.rc = rc
        detail = _lib.load().gbla_last_error().decode() if rc == 1002 else ""
        super().__init__("%s failed: %d (%s) %s" % (name, rc, _lib.status_string(rc), detail))


def _check(name, rc):
    if rc != 0:
        raise GblaError(name, rc)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None and t.numel() > 0 else ctypes.c_void_p(0)


def _is_colmajor(A):
    n, m = A.shape
    return A.stride(0) == 1 and (A.stride(1) >= max(1, n) or m <= 1)


def colmajor(A, dtype=None, copy=False):
    """Column-major version of a 2-D tensor (a copy when copy=True or when needed)."""
    dtype = dtype or A.dtype
    if A.dim() == 1:
        A = A.unsqueeze(1)
    if not copy and A.dtype == dtype and _is_colmajor(A):
        return A
    out = torch.empty_strided(A.shape, (1, max(1, A.shape[0])), dtype=dtype, device=A.device)
    out.copy_(A)
    return out


def _ld(A):
    return max(1, A.stride(1)) if A.shape[1] > 1 else max(1, A.shape[0])


def _ws(nbytes, device):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def _require_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("gbla works on CUDA tensors only (no CPU path)")


def set_wait_timeout_ns(ns):
    _lib.load().gbla_set_wait_timeout_ns(int(ns))


def get_wait_timeout_ns():
    return int(_lib.load().gbla_get_wait_timeout_ns())


# ---------------------------------------------------------------------- LU FP64
def lu_factor(A, nb=0):
    """P A = L U (FP64, partial pivoting). Returns (LU, ipiv int32 1-based, info device int32[1])."""
    _require_cuda(A)
    L = _lib.load()
    n = A.shape[0]
    LU = colmajor(A, torch.float64, copy=True)
    ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    ws = _ws(L.gbla_lu_factor_workspace(n, nb), A.device)
    _check("gbla_lu_factor", L.gbla_lu_factor(n, _p(LU), _ld(LU), _p(ipiv), _p(info), nb, _p(ws),
                                              ws.numel(), _stream()))
    return LU, ipiv[:n], info


def lu_solve(LU, ipiv, B, trans=False, info=None):
    """Solve A X = B (or A^t X = B) from lu_factor's output. Returns X (column-major)."""
    _require_cuda(LU, ipiv, B)
    L = _lib.load()
    n = LU.shape[0]
    vec = B.dim() == 1
    X = colmajor(B, torch.float64, copy=True)
    nrhs = X.shape[1]
    info = torch.zeros(1, dtype=torch.int32, device=B.device) if info is None else info
    LUc = colmajor(LU, torch.float64)
    ws = _ws(L.gbla_lu_solve_workspace(n, nrhs), B.device)
    _check("gbla_lu_solve", L.gbla_lu_solve(1 if trans else 0, n, nrhs, _p(LUc), _ld(LUc), _p(ipiv),
                                            _p(X), _ld(X), _p(info), _p(ws), ws.numel(), _stream()))
    return X[:, 0] if vec else X


# -------------------------------------------------------------------- Cholesky
def chol_factor(A, nb=0):
    """A = L L^t (FP64, lower). Returns (matrix with L in its lower triangle, info device int32[1]).
    The strict upper triangle is copied from A and left untouched. nb: outer block width
    (64, 128, 192 or 256; 0 = 64; see tune_chol_nb)."""
    _require_cuda(A)
    L = _lib.load()
    n = A.shape[0]
    F = colmajor(A, torch.float64, copy=True)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check("gbla_chol_factor", L.gbla_chol_factor(n, _p(F), _ld(F), _p(info), int(nb), _stream()))
    return F, info


def chol_solve(Lf, B, info=None):
    """Solve A X = B from chol_factor's output. Returns X (column-major)."""
    _require_cuda(Lf, B)
    L = _lib.load()
    n = Lf.shape[0]
    vec = B.dim() == 1
    X = colmajor(B, torch.float64, copy=True)
    nrhs = X.shape[1]
    info = torch.zeros(1, dtype=torch.int32, device=B.device) if info is None else info
    Lc = colmajor(Lf, torch.float64)
    ws = _ws(L.gbla_chol_solve_workspace(n, nrhs), B.device)
    _check("gbla_chol_solve", L.gbla_chol_solve(n, nrhs, _p(Lc), _ld(Lc), _p(X), _ld(X), _p(info),
                                                _p(ws), ws.numel(), _stream()))
    return X[:, 0] if vec else X


# ------------------------------------------------------------------ mixed path
def lu_factor_mixed(A, prec="bf16", nb=256, F=None):
    """Low-precision LU of fp32(A): returns (F FP32 factors, ipiv, info)."""
    _require_cuda(A)
    L = _lib.load()
    n = A.shape[0]
    Ac = colmajor(A, torch.float64)
    if F is None:
        F = torch.empty_strided((n, n), (1, max(1, n)), dtype=torch.float32, device=A.device)
    ipiv = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    ws = _ws(L.gbla_lu_factor_mixed_workspace(n, nb, p), A.device)
    _check("gbla_lu_factor_mixed",
           L.gbla_lu_factor_mixed(n, _p(Ac), _ld(Ac), _p(F), _ld(F), _p(ipiv), _p(info), p, nb,
                                  _p(ws), ws.numel(), _stream()))
    return F, ipiv[:n], info


def _stats_dict(st):
    return {"outer": st.outer, "inner": st.inner, "converged": bool(st.converged),
            "beta": st.beta, "beta0": st.beta0}


def gmresir(A, F, ipiv, b, tol=1e-14, inner_tol=1e-8, max_outer=10, restart_m=50, restarts=1,
            x=None):
    """GMRES-based refinement of A x = b with the mixed factors. Synchronous.
    b: a vector (returns x, stats dict) or an n x k matrix (every column refined
    on its own, one set-up of the factors; returns X n x k, list of k dicts).
    Raises GblaError on a hard failure, not on non-convergence."""
    _require_cuda(A, F, ipiv, b)
    L = _lib.load()
    n = A.shape[0]
    Ac = colmajor(A, torch.float64)
    Fc = colmajor(F, torch.float32)
    opts = _lib.GmresirOpts(tol, inner_tol, max_outer, restart_m, restarts)
    ws = _ws(L.gbla_gmresir_workspace(n, restart_m), A.device)
    if b.dim() == 2:
        Bc = colmajor(b, torch.float64)
        k = Bc.shape[1]
        X = torch.empty_strided((n, k), (1, max(1, n)), dtype=torch.float64, device=A.device)
        st = (_lib.GmresirStats * max(k, 1))()
        rc = L.gbla_gmresir_solve_nrhs(n, k, _p(Ac), _ld(Ac), _p(Fc), _ld(Fc), _p(ipiv), _p(Bc), _ld(Bc),
                                       _p(X), _ld(X), ctypes.byref(opts), st, _p(ws), ws.numel(),
                                       _stream())
        if rc not in (0, _lib.GBLA_ERR_NOT_CONVERGED):
            raise GblaError("gbla_gmresir_solve_nrhs", rc)
        return X, [_stats_dict(st[j]) for j in range(k)]
    bc = b.reshape(-1).to(torch.float64).contiguous()
    x = torch.empty(max(n, 1), dtype=torch.float64, device=A.device) if x is None else x
    st = _lib.GmresirStats()
    rc = L.gbla_gmresir_solve(n, _p(Ac), _ld(Ac), _p(Fc), _ld(Fc), _p(ipiv), _p(bc), _p(x),
                              ctypes.byref(opts), ctypes.byref(st), _p(ws), ws.numel(), _stream())
    if rc not in (0, _lib.GBLA_ERR_NOT_CONVERGED):
        raise GblaError("gbla_gmresir_solve", rc)
    return x[:n], _stats_dict(st)


def solve_mixed(A, b, prec="bf16", nb=256, **kw):
    """Mixed-precision LU + GMRES-IR. Returns (x, stats). For a 2-D b (n x k) the
    matrix is factored once and every column is refined on its own: x is n x k and
    stats a list of k dicts."""
    F, ipiv, info = lu_factor_mixed(A, prec, nb)
    x, st = gmresir(A, F, ipiv, b, **kw)
    inf = int(info.item())
    for d in (st if isinstance(st, list) else [st]):
        d["info"] = inf
    return x, st


def _krylov(name, A, b, x0, tol, max_iter, restart_m, F, ipiv):
    _require_cuda(A, b, F, ipiv)
    L = _lib.load()
    n = A.shape[0]
    Ac = colmajor(A, torch.float64)
    bc = b.reshape(-1).to(torch.float64).contiguous()
    x = (torch.zeros(max(n, 1), dtype=torch.float64, device=A.device) if x0 is None
         else x0.reshape(-1).to(torch.float64).clone())
    Fc = colmajor(F, torch.float32) if F is not None else None
    opts = _lib.KrylovOpts(tol, max_iter, restart_m)
    st = _lib.KrylovStats()
    ws = _ws(L.gbla_krylov_workspace(n, restart_m), A.device)
    rc = getattr(L, name)(n, _p(Ac), _ld(Ac), _p(bc), _p(x), _p(Fc), _ld(Fc) if Fc is not None else max(1, n),
                          _p(ipiv), ctypes.byref(opts), ctypes.byref(st), _p(ws), ws.numel(), _stream())
    if rc not in (0, _lib.GBLA_ERR_NOT_CONVERGED):
        raise GblaError(name, rc)
    return x[:n], {"iterations": st.iterations, "converged": bool(st.converged),
                   "breakdown": bool(st.breakdown), "relres": st.relres}


def gmres(A, b, x0=None, tol=1e-10, max_iter=1000, restart_m=50, F=None, ipiv=None):
    """Restarted GMRES(restart_m) for A x = b (FP64), optionally left-preconditioned by
    mixed-precision LU factors (F, ipiv from lu_factor_mixed). Returns (x, stats)."""
    return _krylov("gbla_gmres_solve", A, b, x0, tol, max_iter, restart_m, F, ipiv)


def bicgstab(A, b, x0=None, tol=1e-10, max_iter=1000, F=None, ipiv=None):
    """BiCGSTAB for A x = b (FP64), optionally preconditioned by mixed-precision LU
    factors (F, ipiv from lu_factor_mixed). Returns (x, stats)."""
    return _krylov("gbla_bicgstab_solve", A, b, x0, tol, max_iter, 1, F, ipiv)


def chol_factor_mixed(A, prec="fp16x3", nb=256, F=None):
    """Low-precision Cholesky of fp32(A) (A SPD; its lower triangle is read).
    Returns (F FP32: L in the lower triangle, L^t in the strict upper one, info)."""
    _require_cuda(A)
    L = _lib.load()
    n = A.shape[0]
    Ac = colmajor(A, torch.float64)
    if F is None:
        F = torch.empty_strided((n, n), (1, max(1, n)), dtype=torch.float32, device=A.device)
    info = torch.zeros(1, dtype=torch.int32, device=A.device)
    p = PREC[prec] if isinstance(prec, str) else int(prec)
    ws = _ws(L.gbla_chol_factor_mixed_workspace(n, nb, p), A.device)
    _check("gbla_chol_factor_mixed",
           L.gbla_chol_factor_mixed(n, _p(Ac), _ld(Ac), _p(F), _ld(F), _p(info), p, nb, _p(ws),
                                    ws.numel(), _stream()))
    return F, info


def chol_gmresir(A, F, b, tol=1e-14, inner_tol=1e-8, max_outer=10, restart_m=50, restarts=1):
    """GMRES-based refinement with the mixed Cholesky factors (A: the whole SPD
    matrix, FP64). b: a vector or an n x k matrix. Returns (x or X, stats dict or list)."""
    _require_cuda(A, F, b)
    L = _lib.load()
    n = A.shape[0]
    Ac = colmajor(A, torch.float64)
    Fc = colmajor(F, torch.float32)
    vec = b.dim() == 1
    Bc = colmajor(b, torch.float64)
    k = Bc.shape[1]
    X = torch.empty_strided((n, k), (1, max(1, n)), dtype=torch.float64, device=A.device)
    opts = _lib.GmresirOpts(tol, inner_tol, max_outer, restart_m, restarts)
    st = (_lib.GmresirStats * max(k, 1))()
    ws = _ws(L.gbla_gmresir_workspace(n, restart_m), A.device)
    rc = L.gbla_chol_gmresir_solve_nrhs(n, k, _p(Ac), _ld(Ac), _p(Fc), _ld(Fc), _p(Bc), _ld(Bc), _p(X),
                                        _ld(X), ctypes.byref(opts), st, _p(ws), ws.numel(), _stream())
    if rc not in (0, _lib.GBLA_ERR_NOT_CONVERGED):
        raise GblaError("gbla_chol_gmresir_solve_nrhs", rc)
    sts = [_stats_dict(st[j]) for j in range(k)]
    return (X[:, 0], sts[0]) if vec else (X, sts)


def solve_chol_mixed(A, b, prec="fp16x3", nb=256, **kw):
    """Mixed-precision Cholesky + GMRES-IR for SPD A. Returns (x, stats)."""
    F, info = chol_factor_mixed(A, prec, nb)
    x, st = chol_gmresir(A, F, b, **kw)
    inf = int(info.item())
    for d in (st if isinstance(st, list) else [st]):
        d["info"] = inf
    return x, st


def backward_error(A, X, B):
    """Per-column ||B - A X||_inf / (||A||_inf ||X||_inf) on the device (FP64)."""
    _require_cuda(A, X, B)
    L = _lib.load()
    n = A.shape[0]
    Ac = colmajor(A, torch.float64)
    Xc = colmajor(X, torch.float64)
    Bc = colmajor(B, torch.float64)
    nrhs = Xc.shape[1]
    beta = torch.empty(max(nrhs, 1), dtype=torch.float64, device=A.device)
    ws = _ws(L.gbla_backward_error_workspace(n, nrhs), A.device)
    _check("gbla_backward_error",
           L.gbla_backward_error(n, nrhs, _p(Ac), _ld(Ac), _p(Xc), _ld(Xc), _p(Bc), _ld(Bc), _p(beta),
                                 _p(ws), ws.numel(), _stream()))
    return beta[:nrhs]


# ---------------------------------------------------------------------- autograd
def rank_k_update(U, V, alpha=1.0, beta=0.0, C=None):
    """C = alpha * U V^t + beta * C on the device (FP64). U: m x k, V: n x k."""
    _require_cuda(U, V, C)
    L = _lib.load()
    Uc = colmajor(U, torch.float64)
    Vc = colmajor(V, torch.float64)
    m, k = Uc.shape
    n = Vc.shape[0]
    if C is None:
        C = torch.empty_strided((m, n), (1, max(1, m)), dtype=torch.float64, device=U.device)
        beta = 0.0
    _check("gbla_rank_k_update",
           L.gbla_rank_k_update(m, n, k, float(alpha), _p(Uc), _ld(Uc), _p(Vc), _ld(Vc), float(beta),
                                _p(C), _ld(C), _stream()))
    return C


class _Solve(torch.autograd.Function):
    """x = A^{-1} b with the LU (or Cholesky) factors kept for the backward pass:
    gb = A^{-t} g by the transposed solves with the same factors, gA = -gb x^t."""

    @staticmethod
    def forward(ctx, A, b, method):
        vec = b.dim() == 1
        if method == "lu":
            F, ipiv, info = lu_factor(A)
            x = lu_solve(F, ipiv, b)
        elif method == "chol":
            F, info = chol_factor(A)
            ipiv = None
            x = chol_solve(F, b)
        else:
            raise ValueError(method)
        ctx.method = method
        ctx.vec = vec
        ctx.save_for_backward(F, ipiv if ipiv is not None else torch.empty(0, device=A.device), x)
        return x

    @staticmethod
    def backward(ctx, g):
        F, ipiv, x = ctx.saved_tensors
        g = g.contiguous()
        if ctx.method == "lu":
            gb = lu_solve(F, ipiv, g, trans=True)
        else:
            gb = chol_solve(F, g)
        gb2 = gb.unsqueeze(1) if ctx.vec else gb
        x2 = x.unsqueeze(1) if ctx.vec else x
        gA = rank_k_update(gb2, x2, alpha=-1.0)
        return gA, gb, None


def solve(A, b, method="lu"):
    """Differentiable solve of A x = b on the GPU (FP64). method: "lu" or "chol" (A SPD;
    the gradient with respect to A is returned unsymmetrised, -gb x^t)."""
    return _Solve.apply(A, b, method)


# ------------------------------------------------------------- instrumentation
KERNEL_KINDS = _lib.KERNEL_KINDS


def launch_count():
    """Kernels libgbla has launched in this process."""
    return int(_lib.load().gbla_launch_count())


def prof_enable(kinds):
    """Bracket later launch groups of the given kinds (names) with CUDA events."""
    mask = 0
    for k in kinds:
        mask |= 1 << KERNEL_KINDS.index(k)
    _lib.load().gbla_prof_enable(mask)


def prof_reset():
    _lib.load().gbla_prof_reset()


def prof_read(kind):
    """(groups recorded, summed device ms) for one kind."""
    c = ctypes.c_int(0)
    t = ctypes.c_double(0.0)
    _check("gbla_prof_read", _lib.load().gbla_prof_read(KERNEL_KINDS.index(kind), ctypes.byref(c),
                                                         ctypes.byref(t)))
    return c.value, t.value


def prof_list(kind, max_count=100000):
    """Device ms of each recorded group of one kind, in launch order."""
    buf = (ctypes.c_double * max_count)()
    c = _lib.load().gbla_prof_list(KERNEL_KINDS.index(kind), max_count, buf)
    if c < 0:
        raise GblaError("gbla_prof_list", c)
    return [buf[i] for i in range(c)]


def set_substitution_ctas(ctas):
    """Cap the CTAs of the refinement's substitution (0: one per SM); the
    result does not depend on it."""
    _check("gbla_set_substitution_ctas", _lib.load().gbla_set_substitution_ctas(int(ctas)))


def get_substitution_ctas():
    return int(_lib.load().gbla_get_substitution_ctas())


def set_lookahead(on):
    """Factor the next outer block's panels during the trailing update (same factors)."""
    _check("gbla_set_lookahead", _lib.load().gbla_set_lookahead(1 if on else 0))


def get_lookahead():
    return bool(_lib.load().gbla_get_lookahead())


def fma_peak(precision="fp64", iters=1 << 16):
    """Measured FP64 or FP32 fused multiply-add rate of the current device, TFLOP/s."""
    t = ctypes.c_double(0.0)
    code = {"fp64": 0, "fp32": 1}[precision]
    _check("gbla_fma_peak", _lib.load().gbla_fma_peak(code, int(iters), ctypes.byref(t), _stream()))
    return t.value


# ------------------------------------------------------------------ autotuning
def _tune_nb(kind, n, candidates, run, device, use_cache):
    from . import batched as _b
    key = "%s_nb|%s|%d" % (kind, torch.cuda.get_device_name(device), n)
    cache = _b._load_cache() if use_cache else {}
    if key in cache:
        return cache[key]["nb"]
    res = {}
    for nb in candidates:
        run(nb)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        run(nb)
        e1.record()
        torch.cuda.synchronize()
        res[nb] = e0.elapsed_time(e1)
    best = min(res, key=res.get)
    if use_cache:
        cache[key] = {"nb": best, "candidates_ms": {str(k): v for k, v in res.items()}}
        _b._store_cache(cache)
    return best


def tune_lu_nb(n, candidates=(64, 96, 128, 192, 256), device="cuda", use_cache=True, seed=0):
    """Block size of the FP64 LU for order n, by timing each candidate on a
    uniform random matrix of that order; remembered per GPU and n in the same
    JSON cache as the batched launch shapes."""
    from . import inputs as _in
    A = _in.uniform(n, seed, device)
    return _tune_nb("lu", n, candidates, lambda nb: lu_factor(A, nb=nb), device, use_cache)


def tune_chol_nb(n, candidates=(64, 128, 192, 256), device="cuda", use_cache=True, seed=2):
    """Outer block width of the FP64 Cholesky for order n, timed on an SPD matrix
    B B^t / n + I of that order; cached like tune_lu_nb."""
    from . import inputs as _in
    S = _in.spd(n, seed, device)
    return _tune_nb("chol", n, candidates, lambda nb: chol_factor(S, nb=nb), device, use_cache)
