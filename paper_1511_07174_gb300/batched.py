"""Batched LU (or Cholesky) + solve of many small systems of uneven size (one
persistent launch, replayable as a CUDA graph) and the autotuner that picks
its launch shape.

BatchedLU packs the systems into two flat device buffers (column-major
matrices and right-hand sides), builds the device pointer / size arrays the C
ABI takes (gbla_lu_solve_batched[_f32], or gbla_chol_solve_batched[_f32] with
method="chol"), orders the systems largest first and calls the library. The autotuner times the candidate launch shapes (threads
per CTA x CTAs per SM) on the actual batch and remembers the fastest per GPU,
dtype and batch profile in a JSON cache.
"""
import ctypes
import json
import os

import torch

from . import _lib
from .api import _check, _stream, _ws

CANDIDATES = [(t, c) for t in (128, 256, 512) for c in (1, 2, 4)]


def _cache_path():
    base = os.environ.get("GBLA_CACHE") or os.path.join(
        os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache"), "gbla")
    return os.path.join(base, "autotune.json")


def _load_cache():
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store_cache(cache):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp.%d" % os.getpid()
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


class BatchedLU:
    def __init__(self, As, Bs=None, dtype=torch.float64, device="cuda", method="lu"):
        if method not in ("lu", "chol"):
            raise ValueError("method must be 'lu' or 'chol'")
        self.method = method
        self.dtype = dtype
        self.device = torch.device(device)
        self.sizes = [int(A.shape[0]) for A in As]
        self.nrhs = [int(B.shape[1]) if B.dim() == 2 else 1 for B in Bs] if Bs is not None else None
        if self.nrhs is not None and max(self.nrhs, default=0) > 4:
            raise ValueError("at most 4 right-hand sides per system")
        self.batch = len(As)
        elem = torch.tensor([], dtype=dtype).element_size()
        offA, offB, offP = [], [], []
        ta = tb = tp = 0
        for i, n in enumerate(self.sizes):
            offA.append(ta)
            ta += n * n
            offP.append(tp)
            tp += max(n, 1)
            if self.nrhs is not None:
                offB.append(tb)
                tb += n * self.nrhs[i]
        self.A0 = torch.empty(max(ta, 1), dtype=dtype, device=self.device)
        self.A = torch.empty_like(self.A0)
        self.B0 = torch.empty(max(tb, 1), dtype=dtype, device=self.device)
        self.B = torch.empty_like(self.B0)
        self.ipiv = torch.zeros(max(tp, 1), dtype=torch.int32, device=self.device)
        self.info = torch.zeros(self.batch, dtype=torch.int32, device=self.device)
        flatA = torch.cat([A.t().reshape(-1).to(dtype) for A in As]) if ta else torch.zeros(1, dtype=dtype)
        self.A0[:ta].copy_(flatA)
        if self.nrhs is not None and tb:
            flatB = torch.cat([(B if B.dim() == 2 else B.unsqueeze(1)).t().reshape(-1).to(dtype) for B in Bs])
            self.B0[:tb].copy_(flatB)
        self.offA, self.offB, self.offP = offA, offB, offP
        dev = self.device
        self.d_n = torch.tensor(self.sizes, dtype=torch.int32, device=dev)
        self.d_lda = torch.tensor([max(n, 1) for n in self.sizes], dtype=torch.int32, device=dev)
        self.d_A = torch.tensor([self.A.data_ptr() + o * elem for o in offA], dtype=torch.int64, device=dev)
        self.d_ipiv = torch.tensor([self.ipiv.data_ptr() + o * 4 for o in offP], dtype=torch.int64, device=dev)
        if self.nrhs is not None:
            self.d_nrhs = torch.tensor(self.nrhs, dtype=torch.int32, device=dev)
            self.d_B = torch.tensor([self.B.data_ptr() + o * elem for o in offB], dtype=torch.int64, device=dev)
            self.d_ldb = self.d_lda
        order = sorted(range(self.batch), key=lambda i: -self.sizes[i])
        self.d_order = torch.tensor(order, dtype=torch.int32, device=dev)
        self.max_n = max(self.sizes, default=0)
        L = _lib.load()
        wsf = L.gbla_lu_batched_workspace if method == "lu" else L.gbla_chol_batched_workspace
        self.ws = _ws(wsf(self.batch), dev)
        self.threads, self.ctas_per_sm = 256, 1
        self.graph = None

    # -- execution ---------------------------------------------------------------
    def restore(self):
        """Copy the original matrices and right-hand sides back into the work buffers."""
        self.A.copy_(self.A0)
        self.B.copy_(self.B0)

    def run(self, threads=None, ctas_per_sm=None):
        """Factor and solve every system (one kernel launch on the current stream)."""
        L = _lib.load()
        t = self.threads if threads is None else threads
        c = self.ctas_per_sm if ctas_per_sm is None else ctas_per_sm
        p = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else ctypes.c_void_p(0)
        has_b = self.nrhs is not None
        rhs = (p(self.d_nrhs) if has_b else ctypes.c_void_p(0), p(self.d_B) if has_b else ctypes.c_void_p(0),
               p(self.d_ldb) if has_b else ctypes.c_void_p(0))
        tail = (p(self.info), p(self.d_order), self.max_n, t, c, p(self.ws), self.ws.numel(), _stream())
        if self.method == "lu":
            fn = L.gbla_lu_solve_batched if self.dtype == torch.float64 else L.gbla_lu_solve_batched_f32
            _check("gbla_lu_solve_batched",
                   fn(self.batch, p(self.d_n), p(self.d_A), p(self.d_lda), p(self.d_ipiv), *rhs, *tail))
        else:
            fn = L.gbla_chol_solve_batched if self.dtype == torch.float64 else L.gbla_chol_solve_batched_f32
            _check("gbla_chol_solve_batched",
                   fn(self.batch, p(self.d_n), p(self.d_A), p(self.d_lda), *rhs, *tail))

    def factor(self):
        """Factor every system (factor-only launch): the work buffers hold the
        factors and pivots afterwards, as after run() without right-hand sides."""
        L = _lib.load()
        p = lambda x: ctypes.c_void_p(x.data_ptr()) if x is not None else ctypes.c_void_p(0)
        tail = (p(self.info), p(self.d_order), self.max_n, self.threads, self.ctas_per_sm, p(self.ws),
                self.ws.numel(), _stream())
        f64 = self.dtype == torch.float64
        if self.method == "lu":
            fn = L.gbla_lu_factor_batched if f64 else L.gbla_lu_factor_batched_f32
            _check("gbla_lu_factor_batched", fn(self.batch, p(self.d_n), p(self.d_A), p(self.d_lda),
                                                p(self.d_ipiv), *tail))
        else:
            fn = L.gbla_chol_factor_batched if f64 else L.gbla_chol_factor_batched_f32
            _check("gbla_chol_factor_batched", fn(self.batch, p(self.d_n), p(self.d_A), p(self.d_lda),
                                                  *tail))

    def solve(self, Bs=None):
        """Solve with the factors of an earlier factor() (solve-only launch). Bs: new
        right-hand sides with the same shapes as the constructor's (default: those)."""
        if self.nrhs is None:
            raise ValueError("no right-hand sides")
        if Bs is None:
            self.B.copy_(self.B0)
        else:
            flat = torch.cat([(B if B.dim() == 2 else B.unsqueeze(1)).t().reshape(-1).to(self.dtype)
                              for B in Bs])
            self.B[:flat.numel()].copy_(flat)
        L = _lib.load()
        p = lambda x: ctypes.c_void_p(x.data_ptr())
        tail = (p(self.d_order), self.max_n, self.threads, self.ctas_per_sm, p(self.ws), self.ws.numel(),
                _stream())
        f64 = self.dtype == torch.float64
        if self.method == "lu":
            fn = L.gbla_lu_solve_factored_batched if f64 else L.gbla_lu_solve_factored_batched_f32
            _check("gbla_lu_solve_factored_batched",
                   fn(self.batch, p(self.d_n), p(self.d_A), p(self.d_lda), p(self.d_ipiv), p(self.d_nrhs),
                      p(self.d_B), p(self.d_ldb), *tail))
        else:
            fn = L.gbla_chol_solve_factored_batched if f64 else L.gbla_chol_solve_factored_batched_f32
            _check("gbla_chol_solve_factored_batched",
                   fn(self.batch, p(self.d_n), p(self.d_A), p(self.d_lda), p(self.d_nrhs), p(self.d_B),
                      p(self.d_ldb), *tail))

    def capture(self):
        """Record restore + run as a CUDA graph (after one eager run, so that every
        one-time set-up has happened)."""
        self.restore()
        self.run()
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                self.restore()
                self.run()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    # -- autotuning --------------------------------------------------------------
    def key(self):
        name = torch.cuda.get_device_name(self.device)
        prof = (self.batch, min(self.sizes, default=0), self.max_n, sum(n ** 3 for n in self.sizes) // (1 << 20))
        return "%s|%s|%s|%d|%d|%d|%d" % ((name, self.method, str(self.dtype)) + prof)

    def autotune(self, reps=2, use_cache=True):
        """Time every candidate (threads, CTAs per SM) on this batch; keep the fastest."""
        cache = _load_cache() if use_cache else {}
        k = self.key()
        if k in cache:
            self.threads, self.ctas_per_sm = cache[k]["threads"], cache[k]["ctas_per_sm"]
            return cache[k]
        res = {}
        for t, c in CANDIDATES:
            self.restore()
            self.run(t, c)
            times = []
            for _ in range(reps):
                self.restore()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                self.run(t, c)
                e1.record()
                torch.cuda.synchronize()
                times.append(e0.elapsed_time(e1))
            res["%d,%d" % (t, c)] = min(times)
        best = min(res, key=res.get)
        t, c = (int(v) for v in best.split(","))
        self.threads, self.ctas_per_sm = t, c
        entry = {"threads": t, "ctas_per_sm": c, "ms": res[best], "candidates_ms": res}
        cache[k] = entry
        if use_cache:
            _store_cache(cache)
        return entry

    # -- results -----------------------------------------------------------------
    def results(self):
        """Lists of (LU, ipiv, X) per system as CPU tensors (A[i, j] indexing), and info.
        For method "chol" the first item holds L in its lower triangle (the strict
        upper triangle is the input's) and ipiv is None."""
        A = self.A.cpu()
        B = self.B.cpu()
        P = self.ipiv.cpu()
        out = []
        for i, n in enumerate(self.sizes):
            LU = A[self.offA[i]:self.offA[i] + n * n].reshape(n, n).t()
            piv = P[self.offP[i]:self.offP[i] + n] if self.method == "lu" else None
            X = None
            if self.nrhs is not None:
                k = self.nrhs[i]
                X = B[self.offB[i]:self.offB[i] + n * k].reshape(k, n).t()
            out.append((LU, piv, X))
        return out, self.info.cpu()
