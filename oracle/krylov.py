"""Restarted, left-preconditioned GMRES(m) (Welter & Nguyen, Sec. 3.1 and
Sec. 4.4): Arnoldi with classical (CGS, the paper's setting) or modified
(MGS) Gram-Schmidt, optional second CGS pass (CGS2), Givens rotations on the
Hessenberg matrix and back substitution for the least-squares coefficients.
Test infrastructure: see oracle/__init__.py.

Stopping rule (the paper says only "relative residual norm"; this reading is
shared with the CUDA path): a cycle ends when |g_{j+1}| <= c * rtol *
||P^{-1} b|| (the preconditioned least-squares residual) or after m steps.
At every restart the true residual ||b - K x|| / ||b|| is recomputed; the
solve is accepted when it is <= rtol.  If a cycle ended on the estimate but
the true residual is still too large, c is divided by 10.
"""
import numpy as np


def givens(a, b):
    """Rotation (c, s) with [c s; -s c] [a; b] = [r; 0]."""
    if b == 0.0:
        return 1.0, 0.0
    r = np.hypot(a, b)
    return a / r, b / r


def arnoldi_step(V, w, j, orth):
    """Orthogonalise w against V[:, :j+1]; returns h (j+2,) and the new w."""
    h = np.zeros(j + 2)
    if orth == 'mgs':
        for i in range(j + 1):
            h[i] = V[:, i] @ w
            w = w - h[i] * V[:, i]
    else:
        Vj = V[:, :j + 1]
        h[:j + 1] = Vj.T @ w
        w = w - Vj @ h[:j + 1]
        if orth == 'cgs2':
            h2 = Vj.T @ w
            w = w - Vj @ h2
            h[:j + 1] += h2
    h[j + 1] = np.linalg.norm(w)
    return h, w


def gmres(apply_K, apply_Pinv, b, m=50, rtol=1e-10, maxit=1000, orth='cgs', x0=None):
    """Solve K x = b with left preconditioning P^{-1} K x = P^{-1} b.

    Returns x, info = dict(iters, restarts, true_rel, converged, history).
    """
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros(n), dict(iters=0, restarts=0, true_rel=0.0, converged=True, history=[])
    zb = np.linalg.norm(apply_Pinv(b))
    c = 1.0
    iters = 0
    restarts = 0
    history = []
    r = b - apply_K(x)
    true_rel = np.linalg.norm(r) / bnorm
    while True:
        if true_rel <= rtol:
            return x, dict(iters=iters, restarts=restarts, true_rel=true_rel, converged=True, history=history)
        if iters >= maxit:
            return x, dict(iters=iters, restarts=restarts, true_rel=true_rel, converged=False, history=history)
        z = apply_Pinv(r)
        beta = np.linalg.norm(z)
        V = np.zeros((n, m + 1))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[:, 0] = z / beta
        ended_on_estimate = False
        j_done = 0
        for j in range(m):
            w = apply_Pinv(apply_K(V[:, j]))
            h, w = arnoldi_step(V, w, j, orth)
            iters += 1
            if h[j + 1] > 0.0:
                V[:, j + 1] = w / h[j + 1]
            # apply the previous rotations to the new column, then a new one
            for i in range(j):
                t = cs[i] * h[i] + sn[i] * h[i + 1]
                h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1]
                h[i] = t
            cs[j], sn[j] = givens(h[j], h[j + 1])
            h[j] = cs[j] * h[j] + sn[j] * h[j + 1]
            h[j + 1] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            H[:j + 2, j] = h[:j + 2]
            j_done = j + 1
            history.append(abs(g[j + 1]) / zb)
            if abs(g[j + 1]) <= c * rtol * zb or h[j] == 0.0 or iters >= maxit:
                ended_on_estimate = abs(g[j + 1]) <= c * rtol * zb
                break
        # back substitution with the triangular R = H[:j_done, :j_done]
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:j_done] @ y[i + 1:]) / H[i, i]
        x = x + V[:, :j_done] @ y
        restarts += 1
        r = b - apply_K(x)
        true_rel = np.linalg.norm(r) / bnorm
        if ended_on_estimate and true_rel > rtol:
            c *= 0.1
