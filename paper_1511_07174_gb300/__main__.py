"""Solve one synthetic dense system on the GPU and print the outcome as JSON.

    python -m paper_1511_07174_gb300 [--n 8192] [--kappa 1e4] [--prec fp16x3] [--nb 256]
                                     [--method mixed|lu|chol] [--matrix haar|uniform]

The matrix is A = U diag(s) V^t with Haar-distributed U, V and singular values
spaced geometrically down to 1/kappa, or (--matrix uniform) iid U[-1, 1]
entries (for --method chol: A = B B^t / n + I),
x_true ~ N(0, 1), b = A x_true. `mixed` factors in low precision and refines
with GMRES to backward error 1e-14; `lu` and `chol` are the FP64 paths.
"""
import argparse
import json

import torch

from . import api, inputs


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--kappa", type=float, default=1e4)
    ap.add_argument("--prec", default="fp16x3")
    ap.add_argument("--nb", type=int, default=256)
    ap.add_argument("--method", default="mixed", choices=["mixed", "lu", "chol"])
    ap.add_argument("--matrix", default="haar", choices=["haar", "uniform"])
    args = ap.parse_args()
    dev = "cuda"
    if args.method == "chol":
        A = inputs.spd(args.n, seed=0, device=dev)
    elif args.matrix == "uniform":
        A = inputs.uniform(args.n, seed=0, device=dev)
    else:
        A = inputs.haar_kappa(args.n, args.kappa, device=dev)
    b = A @ inputs.normal((args.n,), 6, dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    if args.method == "mixed":
        x, st = api.solve_mixed(A, b, prec=args.prec, nb=args.nb, max_outer=20)
        out = {k: v for k, v in st.items()}
    elif args.method == "lu":
        LU, ipiv, info = api.lu_factor(A, nb=args.nb)
        x = api.lu_solve(LU, ipiv, b)
        out = {"info": int(info.item())}
    else:
        L, info = api.chol_factor(A)
        x = api.chol_solve(L, b)
        out = {"info": int(info.item())}
    e1.record()
    torch.cuda.synchronize()
    out["beta"] = float(api.backward_error(A, x.reshape(-1, 1), b.reshape(-1, 1))[0].item())
    out["ms"] = e0.elapsed_time(e1)
    out.update(n=args.n, method=args.method, matrix=args.matrix if args.method != "chol" else "spd")
    print(json.dumps(out))


if __name__ == "__main__":
    main()
