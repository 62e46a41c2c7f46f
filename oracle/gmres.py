"""GMRES and GMRES-based iterative refinement, plain numpy FP64 (test infrastructure only).

GMRES (paper section 2): build an orthonormal Krylov basis with (modified)
Gram-Schmidt, keep the Hessenberg matrix in upper-triangular form with Givens
rotations so that the residual norm of the least-squares problem is known at
every step, and restart after a fixed number of steps from the current
iterate.

GMRES-IR: x0 from the low-precision factors; then repeatedly r = b - A x in
FP64, stop when ||r||_inf / (||A||_inf ||x||_inf) <= tol, otherwise solve the
correction equation with GMRES on the left-preconditioned system
M^{-1} A d = M^{-1} r (M = the low-precision factorisation applied in FP64
arithmetic) and update x <- x + d in FP64.

A library matrix-vector product (numpy @) serves as a step where the
algorithm calls for one.
"""
import numpy as np


def gmres(apply_op, rhs, m, tol, restarts=1, x0=None):
    """Restarted GMRES(m) for op(d) = rhs.

    apply_op : callable v -> op(v) (float64 vector in, float64 vector out)
    rhs      : right-hand side
    m        : restart length (Krylov steps per cycle)
    tol      : stop when the least-squares residual <= tol * ||rhs||_2
    restarts : number of cycles
    Returns (d, total_steps, residual_history) where residual_history[k] is
    the estimated ||rhs - op(d_k)||_2 after step k (index 0 = start).
    """
    rhs = np.asarray(rhs, dtype=np.float64)
    n = rhs.shape[0]
    d = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    bnorm = np.linalg.norm(rhs)
    hist = []
    steps = 0
    if bnorm == 0.0:
        return d, 0, [0.0]
    for _cycle in range(restarts):
        r = rhs - apply_op(d) if steps > 0 or x0 is not None else rhs.copy()
        beta = np.linalg.norm(r)
        if not hist:
            hist.append(beta)
        if beta <= tol * bnorm:
            break
        V = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = r / beta
        k = 0
        for j in range(m):
            w = apply_op(V[:, j])
            # modified Gram-Schmidt against v_0..v_j
            for i in range(j + 1):
                H[i, j] = V[:, i] @ w
                w = w - H[i, j] * V[:, i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[:, j + 1] = w / H[j + 1, j]
            # previous rotations on the new column
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            # new rotation zeroing H[j+1, j]
            rho = np.hypot(H[j, j], H[j + 1, j])
            if rho == 0.0:
                cs[j], sn[j] = 1.0, 0.0
            else:
                cs[j], sn[j] = H[j, j] / rho, H[j + 1, j] / rho
            H[j, j] = rho
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            steps += 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= tol * bnorm or H[j, j] == 0.0:
                break
        # back substitution with the k x k upper triangle
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            s = g[i]
            for t in range(i + 1, k):
                s -= H[i, t] * y[t]
            y[i] = s / H[i, i]
        d = d + V[:, :k] @ y
        if hist[-1] <= tol * bnorm:
            break
    return d, steps, hist


def arnoldi(apply_op, v0, k):
    """k steps of Arnoldi with modified Gram-Schmidt: returns (V n x (k+1), H (k+1) x k)."""
    n = v0.shape[0]
    V = np.zeros((n, k + 1))
    H = np.zeros((k + 1, k))
    V[:, 0] = v0 / np.linalg.norm(v0)
    for j in range(k):
        w = apply_op(V[:, j])
        for i in range(j + 1):
            H[i, j] = V[:, i] @ w
            w = w - H[i, j] * V[:, i]
        H[j + 1, j] = np.linalg.norm(w)
        V[:, j + 1] = w / H[j + 1, j]
    return V, H


def inf_backward_error(A, x, b, anorm=None):
    """||b - A x||_inf / (||A||_inf ||x||_inf), FP64."""
    if anorm is None:
        anorm = np.abs(A).sum(axis=1).max()
    r = b - A @ x
    den = anorm * np.abs(x).max()
    return float(np.abs(r).max() / den) if den > 0 else float("inf")


def gmres_ir(A, b, apply_minv, tol=1e-14, m=50, tau=1e-8, max_outer=10, restarts=1):
    """GMRES-based iterative refinement.

    A          : float64 n x n
    b          : float64 vector
    apply_minv : callable v -> M^{-1} v (the low-precision factors, FP64 arithmetic)
    Returns (x, info dict with outer, inner_total, beta_history, converged).
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    anorm = np.abs(A).sum(axis=1).max()
    x = apply_minv(b)
    betas = []
    inner_total = 0
    converged = False
    outer = 0
    while True:
        r = b - A @ x
        xn = np.abs(x).max()
        beta = float(np.abs(r).max() / (anorm * xn)) if xn > 0 else float("inf")
        betas.append(beta)
        if beta <= tol:
            converged = True
            break
        if outer >= max_outer:
            break
        z = apply_minv(r)
        d, steps, _ = gmres(lambda v: apply_minv(A @ v), z, m, tau, restarts=restarts)
        inner_total += steps
        x = x + d
        outer += 1
    return x, {"outer": outer, "inner_total": inner_total, "beta_history": betas,
               "converged": converged}


def bicgstab(A, b, tol, max_iter, x0=None, apply_minv=None):
    """BiCGSTAB (the stabilised BiCG of paper section 2), plain numpy FP64,
    written from the method's recurrences (van der Vorst's form, with the
    preconditioner applied to the search directions: p^ = M^{-1} p,
    s^ = M^{-1} s; no preconditioner when apply_minv is None):

        r = b - A x,  r~ = r,  rho = alpha = omega = 1,  v = p = 0
        repeat:
          rho' = (r~, r);  beta = (rho' / rho) (alpha / omega)
          p = r + beta (p - omega v);  p^ = M^{-1} p;  v = A p^
          alpha = rho' / (r~, v);  s = r - alpha v
          s^ = M^{-1} s;  t = A s^;  omega = (t, s) / (t, t)
          x = x + alpha p^ + omega s^;  r = s - omega t;  rho = rho'
        until ||r||_2 <= tol ||b||_2 or max_iter iterations.

    When t = A s^ vanishes, x + alpha p^ is taken: it is the solution when
    s = 0, otherwise the method broke down.
    Returns (x, info dict: iterations, converged, relres history (index 0 =
    start), breakdown flag when rho' vanishes or t does with s != 0)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    minv = apply_minv if apply_minv is not None else (lambda v: np.array(v, dtype=np.float64))
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - A @ x
    rt = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros(n)
    p = np.zeros(n)
    bnorm = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / bnorm if bnorm > 0 else 0.0]
    it = 0
    breakdown = False
    converged = hist[0] <= tol
    while not converged and it < max_iter:
        rho_new = rt @ r
        if rho_new == 0.0:
            breakdown = True
            break
        beta = (rho_new / rho) * (alpha / omega)
        p = r + beta * (p - omega * v)
        ph = minv(p)
        v = A @ ph
        alpha = rho_new / (rt @ v)
        s = r - alpha * v
        sh = minv(s)
        t = A @ sh
        tt = t @ t
        if tt == 0.0:
            # t = 0: s = 0 (x + alpha p^ solves the system) or a breakdown
            x = x + alpha * ph
            r = s
            it += 1
            hist.append(np.linalg.norm(r) / bnorm)
            converged = hist[-1] <= tol
            breakdown = not converged
            break
        omega = (t @ s) / tt
        x = x + alpha * ph + omega * sh
        r = s - omega * t
        rho = rho_new
        it += 1
        hist.append(np.linalg.norm(r) / bnorm)
        converged = hist[-1] <= tol
    return x, {"iterations": it, "converged": converged, "relres": hist, "breakdown": breakdown}
