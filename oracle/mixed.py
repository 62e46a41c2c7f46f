"""Low-precision blocked LU, plain numpy (test infrastructure only).

The method's mixed-precision factorisation written out step by step: the
working matrix is held in FP32; the LU is right-looking and blocked ("delayed
updating", paper section 2: nb rank-1 updates replaced by one rank-nb update).
Per block column:
  1. the panel W[k0:, k0:k0+nb] is factored by partial pivoting (paper
     section 2), FP64 arithmetic, each stored value rounded to FP32; its row
     interchanges are applied across whole rows;
  2. U12 = L11^{-1} W12 by forward substitution (FP64 arithmetic, stored FP32);
  3. W22 <- W22 - L21 U12, where the product takes its operands rounded to the
     update precision and accumulates in FP32:
       fp32 -- operands as stored;
       tf32 -- operands rounded to 10 mantissa bits, nearest, ties away;
       bf16 / fp16 -- each row of L21 and each column of U12 multiplied by a
         power of two 2^e chosen so that its largest magnitude lies in
         [2^14, 2^15), then rounded to nearest-even in the 16-bit format; the
         FP32 product is multiplied by 2^-(e_row + e_col), which is exact;
       fp16x3 / bf16x3 -- the scaled operands split as hi + lo (hi rounded,
         lo = rounded remainder) and the product taken as
         hi*hi + hi*lo + lo*hi in one FP32 accumulation.
A library matrix product (numpy float32 @) serves as step 3's product.
"""
import numpy as np

SCALE_TOP = 15      # largest magnitude of a scaled sliver lies in [2^(T-1), 2^T)
SCALE_CLAMP = 100   # |e| is clamped so that 2^e stays a normal FP32 number


def to_fp32(x):
    return np.asarray(x, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_tf32(x32):
    """Round FP32 values to TF32 (10 explicit mantissa bits), nearest, ties away from zero."""
    a = np.ascontiguousarray(np.asarray(x32, dtype=np.float32))
    bits = a.view(np.uint32).copy()
    finite = np.isfinite(a)
    rb = (bits + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    bits = np.where(finite, rb, bits)
    return bits.view(np.float32).astype(np.float64)


def round_bf16(x32):
    """Round FP32 values to bfloat16, nearest-even (bit arithmetic on the FP32 pattern)."""
    a = np.ascontiguousarray(np.asarray(x32, dtype=np.float32))
    bits = a.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rb = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    out = (rb & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    out = np.where(np.isfinite(a), out, a.view(np.uint32))
    return out.view(np.float32).astype(np.float64)


def round_fp16(x32):
    return np.asarray(x32, dtype=np.float32).astype(np.float16).astype(np.float64)


def sliver_exponent(maxabs):
    """e with maxabs * 2^e in [2^(T-1), 2^T), clamped; 0 for an all-zero sliver."""
    maxabs = np.asarray(maxabs, dtype=np.float64)
    _, E = np.frexp(maxabs)
    e = np.where(maxabs > 0, SCALE_TOP - E, 0)
    return np.clip(e, -SCALE_CLAMP, SCALE_CLAMP).astype(np.int64)


def lowprec_product(L21, U12, prec):
    """FP32-accumulated product L21 @ U12 with operands in the update precision."""
    if prec == "fp32":
        a, b = L21, U12
        return (a.astype(np.float32) @ b.astype(np.float32)).astype(np.float64)
    if prec == "tf32":
        a, b = round_tf32(L21), round_tf32(U12)
        return (a.astype(np.float32) @ b.astype(np.float32)).astype(np.float64)
    if prec in ("bf16", "fp16"):
        rnd = round_bf16 if prec == "bf16" else round_fp16
        ea = sliver_exponent(np.abs(L21).max(axis=1) if L21.shape[1] else np.zeros(L21.shape[0]))
        eb = sliver_exponent(np.abs(U12).max(axis=0) if U12.shape[0] else np.zeros(U12.shape[1]))
        a = rnd(np.ldexp(L21, ea[:, None]))
        b = rnd(np.ldexp(U12, eb[None, :]))
        d = (a.astype(np.float32) @ b.astype(np.float32)).astype(np.float64)
        return np.ldexp(d, -(ea[:, None] + eb[None, :]))
    if prec in ("fp16x3", "bf16x3"):
        rnd = round_bf16 if prec == "bf16x3" else round_fp16
        ea = sliver_exponent(np.abs(L21).max(axis=1) if L21.shape[1] else np.zeros(L21.shape[0]))
        eb = sliver_exponent(np.abs(U12).max(axis=0) if U12.shape[0] else np.zeros(U12.shape[1]))
        a = to_fp32(np.ldexp(L21, ea[:, None]))
        b = to_fp32(np.ldexp(U12, eb[None, :]))
        ahi = rnd(a)
        alo = rnd(a - ahi)
        bhi = rnd(b)
        blo = rnd(b - bhi)
        # one FP32-accumulated product over the concatenated K: hi*hi + hi*lo + lo*hi
        A3 = np.concatenate([ahi, ahi, alo], axis=1).astype(np.float32)
        B3 = np.concatenate([bhi, blo, bhi], axis=0).astype(np.float32)
        d = (A3 @ B3).astype(np.float64)
        return np.ldexp(d, -(ea[:, None] + eb[None, :]))
    raise ValueError(prec)


def lu_lowprec(A, nb, prec, with_gap=False, force_ipiv=None, ko=None):
    """Blocked right-looking GEPP of fp32(A). Returns (W packed L\\U as FP32 values in float64,
    ipiv int32 1-based, info), and with with_gap=True also the smallest relative
    gap (|a_p| - |a_second|) / |a_p| between the two largest candidates of any
    pivot search (1.0 when no column has two candidates) -- the diagnostic that
    tells whether a second elimination with slightly different rounding must
    choose the same pivots.

    force_ipiv (1-based, as returned): take these pivots instead of searching
    (another implementation's choices); the extra return value is then the
    largest relative shortfall (max|a| - |a_forced|) / max|a| of a forced pivot
    against the column's largest candidate (0.0 when every forced pivot is a
    largest candidate).

    ko (a multiple of nb): two-level delayed updating (paper section 2's k
    rank-1 updates replaced by one rank-k update, applied twice). Within a
    super-block of ko columns every nb-block is factored and updates only the
    super-block's own columns; then the super-block's rows of the columns
    right of it are solved block by block (each block's FP32 substitution,
    then the update of the super-block's rows below it in the update
    precision), and the rows below the super-block receive one rank-ko update
    with operand scales over the whole ko-long slivers."""
    W = to_fp32(np.array(A, dtype=np.float64, order="F"))
    n = W.shape[0]
    ipiv = np.zeros(n, dtype=np.int32)
    info = 0
    gap = 1.0
    slack = 0.0
    ko = nb if ko is None else ko
    if ko % nb != 0:
        raise ValueError("ko must be a multiple of nb")
    for K0 in range(0, n, ko):
        E = min(K0 + ko, n)
        for k0 in range(K0, E, nb):
            k1 = min(k0 + nb, E)
            # 1. panel, unblocked, FP64 arithmetic rounded to FP32
            for j in range(k0, k1):
                col = np.abs(W[j:, j])
                if force_ipiv is not None:
                    p = int(force_ipiv[j]) - 1
                    if col.max() > 0:
                        slack = max(slack, float((col.max() - col[p - j]) / col.max()))
                else:
                    p = j + int(np.argmax(col))          # first maximum -> lowest index
                if col.shape[0] > 1 and col.max() > 0:
                    top2 = np.sort(col)[-2:]
                    gap = min(gap, float((top2[1] - top2[0]) / top2[1]))
                ipiv[j] = p + 1
                if W[p, j] != 0.0:
                    if p != j:
                        W[[j, p], :] = W[[p, j], :]
                    W[j + 1:, j] = to_fp32(W[j + 1:, j] / W[j, j])
                elif info == 0:
                    info = j + 1
                if j + 1 < k1:
                    W[j + 1:, j + 1:k1] = to_fp32(W[j + 1:, j + 1:k1]
                                                 - np.outer(W[j + 1:, j], W[j, j + 1:k1]))
            if k1 >= E:
                continue
            # 2. U12 = L11^{-1} W12 for the super-block's columns right of the
            #    block, forward substitution with unit diagonal
            for j in range(k0, k1):
                if j + 1 < k1:
                    W[j + 1:k1, k1:E] = to_fp32(W[j + 1:k1, k1:E] - np.outer(W[j + 1:k1, j], W[j, k1:E]))
            # 3. update of those columns, all rows below the block, in the update precision
            D = lowprec_product(W[k1:, k0:k1], W[k0:k1, k1:E], prec)
            W[k1:, k1:E] = (W[k1:, k1:E].astype(np.float32) - D.astype(np.float32)).astype(np.float64)
        if E >= n:
            break
        # 4. the super-block's rows of the columns right of it, block by block
        for k0 in range(K0, E, nb):
            k1 = min(k0 + nb, E)
            for j in range(k0, k1):
                if j + 1 < k1:
                    W[j + 1:k1, E:] = to_fp32(W[j + 1:k1, E:] - np.outer(W[j + 1:k1, j], W[j, E:]))
            if k1 < E:
                D = lowprec_product(W[k1:E, k0:k1], W[k0:k1, E:], prec)
                W[k1:E, E:] = (W[k1:E, E:].astype(np.float32) - D.astype(np.float32)).astype(np.float64)
        # 5. one rank-(E - K0) update of the rows below the super-block
        D = lowprec_product(W[E:, K0:E], W[K0:E, E:], prec)
        W[E:, E:] = (W[E:, E:].astype(np.float32) - D.astype(np.float32)).astype(np.float64)
    if force_ipiv is not None:
        return W, ipiv, info, slack
    if with_gap:
        return W, ipiv, info, gap
    return W, ipiv, info


def apply_minv_factory(W, ipiv):
    """M^{-1} v = U^{-1} L^{-1} P v with the FP32-valued factors, FP64 arithmetic (plain loops
    over columns; numpy slices as the inner loops)."""
    n = W.shape[0]
    Lc = np.tril(W, -1)
    Uc = np.triu(W)

    def apply(v):
        b = np.array(v, dtype=np.float64)
        for j in range(n):
            p = int(ipiv[j]) - 1
            if p != j:
                b[j], b[p] = b[p], b[j]
        for j in range(n):
            b[j + 1:] -= Lc[j + 1:, j] * b[j]
        for j in range(n - 1, -1, -1):
            b[j] = b[j] / Uc[j, j]
            b[:j] -= Uc[:j, j] * b[j]
        return b

    return apply


def chol_lowprec(A, nb, prec):
    """Blocked right-looking Cholesky A = L L^t of fp32(A), lower triangle
    (paper section 2 for SPD systems), in the mixed precision of lu_lowprec.
    Per block column k0 .. k1:
      1. the diagonal block, column by column: d = a_jj, d <= 0 stops with
         info = j + 1; l_jj = sqrt(d); l_ij = a_ij / l_jj; a_ik -= l_ij l_kj
         inside the block -- FP64 arithmetic, each stored value rounded to FP32;
      2. the rows below it, L21 = A21 L11^{-t}, by substitution column by
         column (FP64 arithmetic, stored FP32);
      3. the trailing lower triangle A22 -= L21 L21^t with lowprec_product
         (the same operand rounding and scaling as the LU's update; the row
         scale of L21 serves both factors).
    Returns (W with L in its lower triangle, FP32 values in float64; the
    strict upper triangle is not meaningful), info."""
    W = to_fp32(np.array(A, dtype=np.float64, order="F"))
    n = W.shape[0]
    for k0 in range(0, n, nb):
        k1 = min(k0 + nb, n)
        for j in range(k0, k1):
            d = W[j, j]
            if not d > 0.0:
                return W, j + 1
            W[j, j] = to_fp32(np.sqrt(d))
            W[j + 1:k1, j] = to_fp32(W[j + 1:k1, j] / W[j, j])
            if j + 1 < k1:
                # lower part of the rest of the diagonal block
                upd = np.tril(np.outer(W[j + 1:k1, j], W[j + 1:k1, j]))
                W[j + 1:k1, j + 1:k1] = to_fp32(W[j + 1:k1, j + 1:k1] - upd)
        if k1 >= n:
            break
        # 2. L21 = A21 L11^{-t}: column j of L21 = (A21[:, j] - sum_{k<j} L21[:, k] l_jk) / l_jj
        for j in range(k0, k1):
            s = W[k1:, j].copy()
            for k in range(k0, j):
                s = s - W[k1:, k] * W[j, k]
            W[k1:, j] = to_fp32(s / W[j, j])
        # 3. trailing lower triangle
        L21 = W[k1:, k0:k1]
        D = lowprec_product(L21, L21.T.copy(), prec)
        W22 = (W[k1:, k1:].astype(np.float32) - D.astype(np.float32)).astype(np.float64)
        W[k1:, k1:] = np.tril(W22) + np.triu(W[k1:, k1:], 1)
    return W, 0


def chol_minv_factory(W):
    """M^{-1} v = L^{-t} L^{-1} v with the FP32-valued factor (lower triangle of
    W), FP64 arithmetic: forward substitution with L, back substitution with
    L^t."""
    n = W.shape[0]
    Lc = np.tril(W)

    def apply(v):
        b = np.array(v, dtype=np.float64)
        for j in range(n):
            b[j] = b[j] / Lc[j, j]
            b[j + 1:] -= Lc[j + 1:, j] * b[j]
        for j in range(n - 1, -1, -1):
            b[j] = (b[j] - Lc[j + 1:, j] @ b[j + 1:]) / Lc[j, j]
        return b

    return apply
