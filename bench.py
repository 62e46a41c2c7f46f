"""Benchmark: dense LU solve at n = 16384, mixed precision + GMRES-IR vs FP64.

Workload (synthetic): three n x n systems A x = b with A = U diag(s) V^t, U, V
Haar orthogonal (QR of Gaussian, seeds 4 and 5), s geometric from 1 to
1/kappa for kappa in {1e2, 1e4, 1e6}, x_true ~ N(0, 1) (seed 6), b = A x_true.
One step = solve all three to normwise backward error <= 1e-14: low-precision
LU (FP32 working matrix, tensor-core trailing update) + GMRES-based iterative
refinement in FP64. Metric: TFLOP/s counted as 2/3 n^3 per solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). Inputs (2 GiB FP64 per matrix) are larger than
the 129 MB L2, so no flush is needed between steps. Under torchrun every rank
runs its own replica of the workload (the solver does not shard: replicas only)
and the value is the work of all ranks over the slowest rank's time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "LU solve TFLOP/s (2/3n^3) n=16384: mixed+GMRES-IR vs FP64 at 1e-14 bkwd err"
KAPPAS = (1e2, 1e4, 1e6)
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (DFMA) nominal; the FP64 GEMM is measured against it


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", "--matrix-size", dest="n", type=int, default=16384)
    ap.add_argument("--prec", default="fp16x3")
    ap.add_argument("--nb", type=int, default=256)
    ap.add_argument("--restart", type=int, default=50)
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--e2e-warmup", type=int, default=1,
                    help="untimed end-to-end steps first (the first copy from freshly pinned "
                         "host buffers maps their pages and runs at a fraction of the link rate)")
    ap.add_argument("--streams", type=int, default=3,
                    help="systems of a step solved concurrently, each on its own CUDA stream "
                         "and host thread (1: one after the other)")
    ap.add_argument("--subst-ctas", type=int, default=0,
                    help="cap on the CTAs of the refinement's substitution (0: one per SM)")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the other workloads (FP64 LU/Cholesky n=8192, batched, autograd)")
    ap.add_argument("--cpu-ksteps", type=int, default=8,
                    help="elimination steps of the oracle sample (bounded CPU baseline)")
    return ap.parse_args()


# ----------------------------------------------------------------- distributed
def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return ws, rank


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, ws):
    if ws == 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# --------------------------------------------------------------------- helpers
def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return dict(FALLBACK_PEAKS), "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while active."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_workload(n, device):
    from paper_1511_07174_gb300 import inputs
    U = inputs.haar(n, 4, device)
    V = inputs.haar(n, 5, device)
    x_true = inputs.normal((n,), 6, device)
    As, bs = [], []
    for kappa in KAPPAS:
        A = inputs.haar_kappa(n, kappa, UV=(U, V), device=device)
        As.append(A)
        bs.append(A @ x_true)
    del U, V
    torch.cuda.synchronize() if device != "cpu" else None
    return As, bs, x_true


def lu_flops(n):
    return 2.0 / 3.0 * float(n) ** 3


def gemm_tc_algorithmic_flops(n, nb):
    """2 * M * N * K summed over the trailing updates of the blocked LU."""
    tot = 0.0
    for k0 in range(0, n, nb):
        kb = min(nb, n - k0)
        nt = n - k0 - kb
        if nt > 0:
            tot += 2.0 * nt * nt * kb
    return tot


def panel_algorithmic_bytes(n, elem, nb):
    """Each panel launch reads and writes its slab (32 columns, rows k..n) once, and
    reads and writes the two rows of each of its (at most 32) interchanges in the
    other columns of its outer block (nb - 32 of them)."""
    tot = 0.0
    for j0 in range(0, n, 32):
        w = min(32, n - j0)
        k0 = (j0 // nb) * nb
        others = min(nb, n - k0) - w
        tot += 2.0 * (n - j0) * w * elem
        tot += 2.0 * 2.0 * w * others * elem
    return tot


def trsv_algorithmic_bytes(n, elem):
    """One triangular solve reads its triangle once (n(n+1)/2 elements) plus the vector."""
    return n * (n + 1) / 2.0 * elem + 2.0 * n * 8


def oracle_sample(A_host, ksteps):
    """Time the CPU oracle on the first `ksteps` elimination steps of the n x n matrix."""
    import oracle
    n = A_host.shape[0]
    t0 = time.perf_counter()
    oracle.getrf(A_host, ksteps=ksteps)
    dt = time.perf_counter() - t0
    flops = 0.0
    for j in range(ksteps):
        m = n - j - 1
        flops += m + 2.0 * m * m
    return flops, dt


# ---------------------------------------------------------------- reference arm
def bench_config(args, nsys, ws):
    """The workload both arms are quoted on."""
    n = args.n
    return {"workload": "dense LU solve n=%d, 3 systems (kappa 1e2, 1e4, 1e6; Haar U,V; "
                        "geometric singular values), 1 RHS each, to backward error 1e-14" % n,
            "n": n, "prec": args.prec, "nb": args.nb, "restart": args.restart,
            "systems_per_step": nsys, "parallelism": "replicas" if ws > 1 else "single",
            "l2": "no flush: each FP64 matrix (%.1f GiB) exceeds L2" % (n * n * 8 / 2 ** 30)}


def run_reference(args, ws, rank):
    if rank != 0:
        return
    n = args.n
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    As, bs, _ = make_workload(n, dev)
    A_host = np.asfortranarray(As[1].cpu().numpy())
    del As, bs
    for _ in range(args.warmup):
        oracle_sample(A_host, args.cpu_ksteps)
    times, flops = [], 0.0
    for _ in range(args.steps):
        f, dt = oracle_sample(A_host, args.cpu_ksteps)
        times.append(dt)
        flops = f
    tmean = sum(times) / len(times)
    value = flops / tmean / 1e12
    sample = ("first %d elimination steps of LU with partial pivoting on the n=%d, kappa=1e4 "
              "matrix (%.3g flop), plain FP64 C oracle, 1 thread" % (args.cpu_ksteps, n, flops))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tmean * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, len(KAPPAS), 1),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------- our arm
def solve_one(api, A, b, args, F):
    Fk, ipiv, info = api.lu_factor_mixed(A, prec=args.prec, nb=args.nb, F=F)
    x, st = api.gmresir(A, Fk, ipiv, b, tol=1e-14, inner_tol=1e-8, max_outer=20,
                        restart_m=args.restart)
    st["x"] = x
    return st


class Concurrent:
    """The systems of a step are independent: each is factored and refined on a
    CUDA stream of its own, issued by a host thread of its own (the refinement
    reads its convergence test on the host, so one thread per system keeps the
    other systems' work queued meanwhile). Every stream starts after the work
    already on the caller's stream, and the caller's stream waits for all of
    them at the end, so events on the caller's stream bracket the whole step."""

    def __init__(self, k):
        self.device = torch.cuda.current_device()
        self.streams = [torch.cuda.Stream() for _ in range(k)]

    def run(self, jobs):
        """Job i runs on stream i mod k; the jobs of one stream run in order on
        one host thread."""
        main = torch.cuda.current_stream()
        k = len(self.streams)
        out = [None] * len(jobs)
        err = []

        def work(t):
            try:
                torch.cuda.set_device(self.device)
                s = self.streams[t]
                s.wait_stream(main)
                with torch.cuda.stream(s):
                    for i in range(t, len(jobs), k):
                        out[i] = jobs[i]()
            except BaseException as e:  # re-raised on the caller's thread
                err.append(e)

        th = [threading.Thread(target=work, args=(t,)) for t in range(min(k, len(jobs)))]
        for t in th:
            t.start()
        for t in th:
            t.join()
        for s in self.streams:
            main.wait_stream(s)
        if err:
            raise err[0]
        return out


def solve_all(api, As, bs, args, Fs, conc=None):
    if conc is None:
        return [solve_one(api, A, b, args, Fs[0]) for A, b in zip(As, bs)]
    jobs = [(lambda A=A, b=b, F=Fs[i % len(Fs)]: solve_one(api, A, b, args, F))
            for i, (A, b) in enumerate(zip(As, bs))]
    return conc.run(jobs)


def run_ours(args, ws, rank):
    from paper_1511_07174_gb300 import api
    import __graft_entry__
    __graft_entry__.build()
    n = args.n
    dev = "cuda"
    As, bs, x_true = make_workload(n, dev)
    nsys = len(As)
    api.set_substitution_ctas(args.subst_ctas)
    nconc = max(1, min(args.streams, nsys))
    Fs = [torch.empty_strided((n, n), (1, n), dtype=torch.float32, device=dev) for _ in range(nconc)]
    conc = Concurrent(nconc) if nconc > 1 else None

    # warm-up; the first warm-up step runs the systems one after the other and
    # records every kernel group (a per-group breakdown without overlap) to
    # find the dominant one
    api.prof_enable(api.KERNEL_KINDS)
    api.prof_reset()
    for w in range(max(args.warmup, 1)):
        solve_all(api, As, bs, args, Fs, None if w == 0 else conc)
        if w == 0:
            torch.cuda.synchronize()
            per_kind = {k: api.prof_read(k) for k in api.KERNEL_KINDS}
            api.prof_reset()
            api.prof_enable([])
    # the dominant group by held SM time (duration x SMs held: a cluster panel
    # holds its 16 SMs, every other kernel group the whole GPU): with the
    # systems concurrent, that is what bounds a step
    nsms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    sm_ms = {k: v[1] * (16 if k == "panel" else nsms) for k, v in per_kind.items()}
    dominant = max(sm_ms, key=lambda k: sm_ms[k])
    fma64 = api.fma_peak("fp64")

    # timed region
    api.prof_enable([dominant])
    api.prof_reset()
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    launches0 = api.launch_count()
    barrier(ws)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    all_stats = []
    for _ in range(args.steps):
        all_stats.append(solve_all(api, As, bs, args, Fs, conc))
    ev1.record()
    torch.cuda.synchronize()
    barrier(ws)
    launches = api.launch_count() - launches0
    clk = clocks.stop()
    ms_total = ev0.elapsed_time(ev1)
    ms_total = max_over_ranks(ms_total, ws)
    ms_step = ms_total / args.steps
    dom_count, dom_ms = api.prof_read(dominant)
    api.prof_enable([])
    value = ws * nsys * lu_flops(n) / (ms_step * 1e-3) / 1e12

    # correctness of the last step: device backward error and independent CPU oracle matvec
    import oracle
    last = all_stats[-1]
    betas_dev = [st["beta"] for st in last]
    betas_oracle = []
    if rank == 0:
        for A, b, st in zip(As, bs, last):
            betas_oracle.append(float(oracle.backward_error(
                np.asfortranarray(A.cpu().numpy()), st["x"].cpu().numpy(), b.cpu().numpy())[0]))

    # FP64 path at kappa = 1e4 (one timed solve after a small warm-up)
    api.lu_factor(As[1][:1024, :1024].contiguous())
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    LU, ipiv, info = api.lu_factor(As[1])
    x64 = api.lu_solve(LU, ipiv, bs[1])
    e1.record()
    torch.cuda.synchronize()
    fp64_ms = e0.elapsed_time(e1)
    fp64_beta = float(api.backward_error(As[1], x64, bs[1]).item())
    del LU, x64

    # end to end through the public API from pinned host buffers
    hostA = [A.cpu().pin_memory() for A in As]
    hostb = [b.cpu().pin_memory() for b in bs]
    dA = [torch.empty_like(A) for A in As]
    db = [torch.empty_like(b) for b in bs]
    hx = [torch.empty(n, dtype=torch.float64).pin_memory() for _ in As]
    del As, bs
    torch.cuda.synchronize()
    barrier(ws)
    # the inputs of system k + 1 travel on a copy stream while system k is solved
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    main = torch.cuda.current_stream()
    copy_s = torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(nsys)]

    def fetch(k):
        with torch.cuda.stream(copy_s):
            dA[k].copy_(hostA[k], non_blocking=True)
            db[k].copy_(hostb[k], non_blocking=True)
            copied[k].record(copy_s)

    def e2e_step_serial():
        copy_s.wait_stream(main)  # after the previous step has read the buffers
        fetch(0)
        for k in range(nsys):
            if k + 1 < nsys:
                fetch(k + 1)
            main.wait_event(copied[k])
            Fk, ipiv, info = api.lu_factor_mixed(dA[k], prec=args.prec, nb=args.nb, F=Fs[0])
            x, st = api.gmresir(dA[k], Fk, ipiv, db[k], tol=1e-14, max_outer=20,
                                restart_m=args.restart)
            hx[k].copy_(x, non_blocking=True)

    # concurrent systems: two sets of device inputs; while one step's systems
    # are solved from one set, the next step's inputs travel into the other on
    # the copy stream (every step's inputs are copied inside the timed region;
    # the first step's copies are exposed)
    if conc is not None:
        dA2 = [dA, [torch.empty_like(x) for x in dA]]
        db2 = [db, [torch.empty_like(x) for x in db]]
        copied2 = [[torch.cuda.Event() for _ in range(nsys)] for _ in range(2)]

    def fetch_set(p):
        copy_s.wait_stream(main)  # the set's last readers (two steps back) have finished
        with torch.cuda.stream(copy_s):
            for k in range(nsys):
                dA2[p][k].copy_(hostA[k], non_blocking=True)
                db2[p][k].copy_(hostb[k], non_blocking=True)
                copied2[p][k].record(copy_s)

    def e2e_job(p, k):
        # on system k's own stream, once its inputs are in: factor, refine, x out
        torch.cuda.current_stream().wait_event(copied2[p][k])
        Fk, ipiv, info = api.lu_factor_mixed(dA2[p][k], prec=args.prec, nb=args.nb, F=Fs[k % nconc])
        x, st = api.gmresir(dA2[p][k], Fk, ipiv, db2[p][k], tol=1e-14, max_outer=20,
                            restart_m=args.restart)
        hx[k].copy_(x, non_blocking=True)

    def e2e_run(nsteps):
        if conc is None:
            for _ in range(nsteps):
                e2e_step_serial()
            return
        fetch_set(0)
        for i in range(nsteps):
            p = i % 2
            if i + 1 < nsteps:
                fetch_set(1 - p)
            conc.run([(lambda k=k, p=p: e2e_job(p, k)) for k in range(nsys)])

    e2e_run(args.e2e_warmup)
    torch.cuda.synchronize()
    t0.record()
    e2e_run(args.e2e_steps)
    t1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(t0.elapsed_time(t1) / args.e2e_steps, ws)
    e2e_value = ws * nsys * lu_flops(n) / (e2e_ms * 1e-3) / 1e12
    h2d = sum(int(h.numel() * h.element_size()) for h in hostA + hostb)
    d2h = sum(int(h.numel() * h.element_size()) for h in hx)

    # roofline of the dominant kernel group
    pk, src = peaks()
    steps_seen = args.steps
    if dominant == "gemm_tc":
        alg = gemm_tc_algorithmic_flops(n, args.nb) * nsys * steps_seen
        achieved = alg / (dom_ms * 1e-3) / 1e12
        peak = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        bound, unit = "tensor", "TFLOP/s"
        per_launch_units = "2*M*N*K of each rank-%d update (the split variant executes 3x on the tensor pipe)" % args.nb
    elif dominant == "gemm_simt" and args.prec == "fp32":
        alg = gemm_tc_algorithmic_flops(n, args.nb) * nsys * steps_seen
        achieved = alg / (dom_ms * 1e-3) / 1e12
        peak, bound, unit = None, "alu", "TFLOP/s"
        per_launch_units = "2*M*N*K"
    elif dominant == "panel":
        alg = panel_algorithmic_bytes(n, 4, args.nb) * nsys * steps_seen
        achieved = alg / (dom_ms * 1e-3) / 1e9
        peak, bound, unit = pk.get("hbm_gbs"), "hbm", "GB/s"
        per_launch_units = ("panel slab read + written once (32 columns x rows, FP32) + the two rows of "
                            "each of its 32 interchanges read + written in the other nb - 32 columns "
                            "of its outer block")
    elif dominant == "trsv":
        # FP64 arithmetic on the FP32 factor: n(n+1)/2 multiply-adds per solve
        alg = n * (n + 1.0) * dom_count
        achieved = alg / (dom_ms * 1e-3) / 1e12
        peak, bound, unit = fma64, "alu", "TFLOP/s"
        src = "measured (this build's FP64 FMA probe on this GPU)"
        per_launch_units = ("one triangular solve: n(n+1)/2 FP64 multiply-adds on the FP32 factor "
                            "(2 flops each); its bytes: the triangle read once, n(n+1)/2 x 4 B")
    else:
        alg = None
        achieved, peak, bound, unit = None, pk.get("hbm_gbs"), "hbm", "GB/s"
        per_launch_units = ""
    # the other large kernel groups, from the first warm-up step (same work as a timed step)
    others = []
    if per_kind.get("gemm_tc", (0, 0.0))[1] > 0:
        alg_tc = gemm_tc_algorithmic_flops(n, args.nb) * nsys
        mult = 3 if args.prec in ("fp16x3", "bf16x3") else 1
        ach = alg_tc / (per_kind["gemm_tc"][1] * 1e-3) / 1e12
        pk_tc = pk.get("bf16_tflops_sustained", pk.get("bf16_tflops"))
        if args.prec == "tf32" and pk_tc:
            pk_tc = pk_tc / 2.0
        others.append({"kernel": "gemm_tc", "bound": "tensor", "achieved": ach, "peak": pk_tc,
                       "unit": "TFLOP/s", "frac": ach / pk_tc if pk_tc else None,
                       "peak_kind": "sustained (the update runs inside a long step)",
                       "executed_on_tensor_pipe_tflops": ach * mult,
                       "algorithmic_units": "2*M*N*K of the method per rank-nb update (the split "
                                            "operands execute it %dx on the tensor pipe)" % mult})
    if per_kind.get("trsv", (0, 0.0))[1] > 0:
        cnt, ms_tr = per_kind["trsv"]
        ach = trsv_algorithmic_bytes(n, 4) * cnt / (ms_tr * 1e-3) / 1e9
        others.append({"kernel": "trsv", "bound": "hbm", "achieved": ach, "peak": pk.get("hbm_gbs"),
                       "unit": "GB/s", "frac": ach / pk.get("hbm_gbs") if pk.get("hbm_gbs") else None,
                       "algorithmic_units": "FP32 triangle read once + vectors, per solve",
                       "note": "FP64 arithmetic of the late blocks and the block chain bound it"})
    if dominant != "panel" and per_kind.get("panel", (0, 0.0))[1] > 0:
        cnt, ms_p = per_kind["panel"]
        ach = panel_algorithmic_bytes(n, 4, args.nb) * nsys / (ms_p * 1e-3) / 1e9
        others.append({"kernel": "panel", "bound": "hbm", "achieved": ach, "peak": pk.get("hbm_gbs"),
                       "unit": "GB/s", "frac": ach / pk.get("hbm_gbs") if pk.get("hbm_gbs") else None,
                       "algorithmic_units": "slab read + written once plus the interchanged rows of "
                                            "its outer block, per launch",
                       "note": "latency-bound: 32 dependent pivot rounds per launch on 16 SMs"})
    roof = {"kernel": dominant, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": (achieved / peak) if (achieved and peak) else None, "traffic": None,
            "peak_source": src, "launch_groups": dom_count, "ms_in_timed_region": dom_ms,
            "algorithmic_units": per_launch_units}
    roof["held_sm_ms_first_warmup_step"] = {k: round(v, 1) for k, v in sm_ms.items() if v > 0}
    prof_path = os.path.join(ROOT, "profiles", "traffic_per_launch.txt")
    if os.path.exists(prof_path):
        with open(prof_path) as f:
            for ln in f:
                f_ = ln.split()
                if len(f_) >= 3 and not ln.startswith("#") and f_[0] == dominant and int(f_[1]) == n:
                    roof["traffic"] = float(f_[2])
                    roof["traffic_unit"] = "bytes per launch"
                    roof["traffic_source"] = " ".join(f_[3:])

    # bounded CPU baseline: the oracle on the first k elimination steps of one system
    cpu = None
    if rank == 0:
        Ah = np.asfortranarray(hostA[1].numpy())
        flops, dt = oracle_sample(Ah, args.cpu_ksteps)
        cpu = {"value": flops / dt / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "sample": "first %d elimination steps of GEPP on the n=%d kappa=1e4 matrix "
                         "(%.3g flop in %.1f s), plain FP64 C, 1 thread" % (args.cpu_ksteps, n, flops, dt)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "%s update, f32 factors, f64 refinement" % args.prec, "data": "synthetic",
            "config": bench_config(args, nsys, ws),
            "concurrent_systems": nconc,
            "substitution_ctas": args.subst_ctas,
            "roofline": roof,
            "roofline_other_kernels": others,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms, "steps": args.e2e_steps,
                    "warmup_steps": args.e2e_warmup,
                    "how": ("every timed step copies its three systems' A and b from pinned host "
                            "buffers and reads each x back; " +
                            ("the systems are solved concurrently and the next step's inputs are "
                             "copied on a copy stream while the current step is solved (the first "
                             "step's copies are exposed)" if conc is not None else
                             "the next system's inputs are copied on a copy stream while the "
                             "current one is solved"))},
            "gpu_launches": int(launches),
            "clocks": clk,
            "fp64_path": {"ms": fp64_ms, "tflops": lu_flops(n) / (fp64_ms * 1e-3) / 1e12,
                          "beta": fp64_beta, "kappa": 1e4,
                          "speedup_mixed_vs_fp64": fp64_ms / (ms_step / nsys)},
            "refinement": [{"kappa": k, "outer": st["outer"], "inner": st["inner"],
                            "beta_device": st["beta"], "beta_oracle": bo}
                           for k, st, bo in zip(KAPPAS, last, betas_oracle)],
            "kernel_ms_first_warmup_step": {k: round(v[1], 3) for k, v in per_kind.items() if v[0]},
        }
        if not args.no_secondary:
            line["secondary"] = secondary(args, pk)
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------ secondary workloads
def _event_ms(fn, reps=1):
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def chol_mixed_vs_fp64(n, args):
    """Time to backward error <= 1e-14 of the SPD system A x = b: fp16x3 Cholesky +
    GMRES-IR against the FP64 Cholesky + solve (both tuned, events on the stream)."""
    from paper_1511_07174_gb300 import api, inputs
    dev = "cuda"
    A = inputs.spd_fp32_product(n, 2, dev)
    b = A @ inputs.normal((n,), 3, dev)
    F = torch.empty_strided((n, n), (1, n), dtype=torch.float32, device=dev)

    def mixed():
        Fk, info = api.chol_factor_mixed(A, prec="fp16x3", nb=256, F=F)
        return api.chol_gmresir(A, Fk, b, tol=1e-14, max_outer=20, restart_m=args.restart)

    mixed()
    api.prof_enable(["gemm_tc", "trsv", "panel"])
    api.prof_reset()
    ms_m = _event_ms(mixed)
    groups = {k: round(api.prof_read(k)[1], 3) for k in ("gemm_tc", "trsv", "panel")}
    api.prof_enable([])
    x, st = mixed()
    beta_m = float(api.backward_error(A, x, b).item())
    nbc = api.tune_chol_nb(min(n, 8192))

    def fp64():
        Lf, info = api.chol_factor(A, nb=nbc)
        return api.chol_solve(Lf, b)

    ms_d = _event_ms(fp64)
    beta_d = float(api.backward_error(A, fp64(), b).item())
    flops = n ** 3 / 3.0
    return {"n": n, "mixed_ms": ms_m, "mixed_tflops": flops / (ms_m * 1e-3) / 1e12,
            "mixed_outer": st["outer"], "mixed_inner": st["inner"], "mixed_beta": beta_m,
            "mixed_kernel_group_ms": groups,
            "fp64_ms": ms_d, "fp64_tflops": flops / (ms_d * 1e-3) / 1e12, "fp64_beta": beta_d,
            "fp64_nb": nbc, "speedup_mixed_vs_fp64": ms_d / ms_m,
            "workload": "A = B B^t/n + I (B iid N(0,1), product in FP32), x_true N(0,1), fp16x3 update"}


def secondary(args, pk):
    """The other measured workloads of the solver (one GPU): FP64 LU n = 512 and
    n = 8192 (16 RHS, block size autotuned), FP64 Cholesky n = 8192, the batched
    solver (4096 systems, FP64 and FP32, CUDA graph, autotuned launch shape) and
    the differentiable solve at n = 4096 with 8 RHS."""
    import oracle
    from paper_1511_07174_gb300 import api, inputs
    from paper_1511_07174_gb300.batched import BatchedLU
    out = {}
    dev = "cuda"
    # FP64 reference rate: cuBLAS DGEMM (a denominator only, not on the solver path)
    a = torch.randn(8192, 8192, dtype=torch.float64, device=dev)
    torch.matmul(a, a)
    ms = _event_ms(lambda: torch.matmul(a, a))
    fp64_peak = 2 * 8192 ** 3 / (ms * 1e-3) / 1e12
    del a
    out["fp64_dgemm_tflops_measured"] = fp64_peak
    # the device's own FMA rates (probe kernels of this library): the denominators
    # of the ALU-bound lines below; DGEMM stays as context
    api.fma_peak("fp64", iters=1 << 14)
    fma64 = api.fma_peak("fp64")
    fma32 = api.fma_peak("fp32")
    out["fma_peak_tflops_measured"] = {"fp64": fma64, "fp32": fma32,
                                       "how": "independent FMA chains on every SM, CUDA events"}
    # n = 512, one RHS, x_true = 1
    n = 512
    A = inputs.uniform(n, 0, dev)
    b = A @ torch.ones(n, dtype=torch.float64, device=dev)
    api.lu_solve(*api.lu_factor(A)[:2], b)
    ms = _event_ms(lambda: api.lu_solve(*api.lu_factor(A)[:2], b), reps=5)
    LU, piv, _ = api.lu_factor(A)
    x = api.lu_solve(LU, piv, b)
    An = np.asfortranarray(A.cpu().numpy())
    LUo, ipo, _ = oracle.getrf(An)
    out["lu_n512"] = {"ms": ms, "beta_oracle": float(oracle.backward_error(An, x.cpu().numpy(), b.cpu().numpy())[0]),
                      "ipiv_equal_oracle": bool(np.array_equal(piv.cpu().numpy(), ipo))}
    # n = 8192 FP64 LU, 16 RHS
    n = 8192
    A = inputs.uniform(n, 0, dev)
    X_true = inputs.normal((n, 16), 1, dev)
    B = A @ X_true
    nb = api.tune_lu_nb(n)
    LU, piv, info = api.lu_factor(A, nb=nb)
    ms_f = _event_ms(lambda: api.lu_factor(A, nb=nb))
    ms_s = _event_ms(lambda: api.lu_solve(LU, piv, B), reps=3)
    X = api.lu_solve(LU, piv, B)
    beta = float(api.backward_error(A, X, B).max().item())
    tf = lu_flops(n) / (ms_f * 1e-3) / 1e12
    out["lu_n8192_fp64"] = {"nb": nb, "factor_ms": ms_f, "tflops": tf, "frac_of_fp64_dgemm": tf / fp64_peak,
                            "frac_of_fp64_fma_peak": tf / fma64,
                            "solve16_ms": ms_s,
                            "solve_gbs": (n * n * 8) / (ms_s * 1e-3) / 1e9, "beta_max": beta}
    del LU, X
    # n = 8192 FP64 Cholesky
    S = inputs.spd(n, 2, dev)
    Xs = inputs.normal((n, 16), 3, dev)
    Bs = S @ Xs
    nbc = api.tune_chol_nb(n)
    F, info = api.chol_factor(S, nb=nbc)
    ms_c = _event_ms(lambda: api.chol_factor(S, nb=nbc))
    Xc = api.chol_solve(F, Bs)
    tfc = n ** 3 / 3.0 / (ms_c * 1e-3) / 1e12
    out["chol_n8192_fp64"] = {"nb": nbc, "factor_ms": ms_c, "tflops": tfc, "frac_of_fp64_dgemm": tfc / fp64_peak,
                              "frac_of_fp64_fma_peak": tfc / fma64,
                              "beta_max": float(api.backward_error(S, Xc, Bs).max().item())}
    del S, F, Xc, A, B
    # mixed-precision Cholesky + GMRES-IR against the FP64 Cholesky, SPD n = 16384
    # (A = B B^t / n + I, the product formed in FP32), one right-hand side
    out["chol_mixed_n16384"] = chol_mixed_vs_fp64(16384, args)
    # batched: 4096 systems n_i in [16, 256], 1-4 RHS, one persistent launch in a CUDA graph
    sizes, nrhs, As, Bs_, Xs_ = inputs.batched(4096, seed=7)
    flops = sum(2.0 / 3.0 * m ** 3 + 2.0 * m * m * k for m, k in zip(sizes, nrhs))
    for dt, name in ((torch.float64, "batched_fp64"), (torch.float32, "batched_fp32")):
        bl = BatchedLU(As, Bs_, dtype=dt)
        tune = bl.autotune()
        bl.capture()
        bl.replay()
        ms_g = _event_ms(bl.replay, reps=3)           # restore copies + the solver launch
        # the solver launch alone (eager, same launch shape), bracketed by events
        bl.restore()
        api.prof_enable(["batched"])
        api.prof_reset()
        bl.run()
        torch.cuda.synchronize()
        cnt, ms_k = api.prof_read("batched")
        api.prof_enable([])
        res, info = bl.results()
        worst = 0.0
        for (LU_, piv_, Xb), Ab, Bb in zip(res[:512], As[:512], Bs_[:512]):
            Ad = np.asfortranarray(Ab.to(dt).to(torch.float64).numpy())
            worst = max(worst, float(oracle.backward_error(Ad, Xb.to(torch.float64).numpy(),
                                                           Bb.to(dt).to(torch.float64).numpy()).max()))
        entry = {"systems": len(sizes), "graph_ms": ms_g, "kernel_ms": ms_k / max(cnt, 1),
                 "systems_per_s": len(sizes) / (ms_k / max(cnt, 1) * 1e-3),
                 "tflops": flops / (ms_k / max(cnt, 1) * 1e-3) / 1e12,
                 "launch_shape": [bl.threads, bl.ctas_per_sm], "autotune_ms": tune.get("ms"),
                 "beta_max_first512": worst}
        if dt == torch.float64:
            entry["frac_of_fp64_dgemm"] = entry["tflops"] / fp64_peak
            entry["frac_of_fp64_fma_peak"] = entry["tflops"] / fma64
        else:
            entry["frac_of_fp32_fma_peak"] = entry["tflops"] / fma32
        out[name] = entry
        del bl
    # batched Cholesky on SPD systems of the same sizes (A_i^t A_i / n_i + I), FP64
    Sp = [(Ab.t() @ Ab) / Ab.shape[0] + torch.eye(Ab.shape[0], dtype=torch.float64) for Ab in As]
    flops_c = sum(1.0 / 3.0 * m ** 3 + 2.0 * m * m * k for m, k in zip(sizes, nrhs))
    bc = BatchedLU(Sp, Bs_, dtype=torch.float64, method="chol")
    bc.autotune()
    bc.capture()
    bc.replay()
    ms_gc = _event_ms(bc.replay, reps=3)
    bc.restore()
    api.prof_enable(["batched"])
    api.prof_reset()
    bc.run()
    torch.cuda.synchronize()
    cnt, ms_kc = api.prof_read("batched")
    api.prof_enable([])
    resc, infoc = bc.results()
    worst = 0.0
    for (_, _, Xb), Ab, Bb in zip(resc[:512], Sp[:512], Bs_[:512]):
        worst = max(worst, float(oracle.backward_error(np.asfortranarray(Ab.numpy()), Xb.numpy(),
                                                       Bb.numpy()).max()))
    kc = ms_kc / max(cnt, 1)
    out["batched_chol_fp64"] = {"systems": len(sizes), "graph_ms": ms_gc, "kernel_ms": kc,
                                "systems_per_s": len(sizes) / (kc * 1e-3),
                                "tflops": flops_c / (kc * 1e-3) / 1e12,
                                "frac_of_fp64_fma_peak": flops_c / (kc * 1e-3) / 1e12 / fma64,
                                "launch_shape": [bc.threads, bc.ctas_per_sm],
                                "info_nonzero": int((infoc != 0).sum()), "beta_max_first512": worst}
    del bc, Sp
    # differentiable solve n = 4096, 8 RHS: forward and backward
    A, b, g = inputs.autograd_problem(4096, 8, device=dev)
    Ar = A.clone().requires_grad_(True)
    br = b.clone().requires_grad_(True)
    x = api.solve(Ar, br)
    (x * g).sum().backward()
    def fwd_bwd():
        Ar.grad = None
        br.grad = None
        xx = api.solve(Ar, br)
        (xx * g).sum().backward()
    ms_fb = _event_ms(fwd_bwd)
    Ar.grad = None
    xx = api.solve(Ar, br)
    loss = (xx * g).sum()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    loss.backward()
    e1.record()
    torch.cuda.synchronize()
    ms_b = e0.elapsed_time(e1)
    nbytes = 4096 * 4096 * 8 * 3    # gA written once + factors read by two triangular solves
    out["autograd_n4096_8rhs"] = {"forward_backward_ms": ms_fb, "backward_ms": ms_b,
                                  "backward_gbs": nbytes / (ms_b * 1e-3) / 1e9,
                                  "backward_frac_of_hbm": nbytes / (ms_b * 1e-3) / 1e9 / pk.get("hbm_gbs", 6800.0)}
    return out


def main():
    args = parse()
    ws, rank = dist_init(args)
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
