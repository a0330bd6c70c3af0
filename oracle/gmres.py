"""Textbook restarted GMRES(m) for the oracle (test infrastructure only).

Saad & Schultz's method, the Krylov solver the paper uses for A x = b
(Sec. 2.2.2): Arnoldi with modified Gram-Schmidt, Givens rotations on the
Hessenberg matrix, least squares by back substitution, restart after m
steps.  The stop test is |g_{j+1}| / ||b||_2 <= tol (the residual norm the
rotations carry), confirmed by the true residual ||b - A x|| / ||b|| at
every restart and at exit.
"""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, tol=1e-8, restart=10, max_iter=1000, x0=None):
    """Returns (x, info) with info = dict(iters, converged, history, rel_residual).

    ``history`` holds |g_{j+1}| / ||b|| after every Arnoldi step, which is the
    residual norm of the iterate that step would produce.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    hist = []
    if bnorm == 0.0:
        return np.zeros(n), dict(iters=0, converged=True, history=hist, rel_residual=0.0)
    iters = 0
    r = b - matvec(x) if x0 is not None else b.copy()
    beta = np.linalg.norm(r)
    rel = beta / bnorm
    while iters < max_iter:
        if rel <= tol:
            return x, dict(iters=iters, converged=True, history=hist, rel_residual=rel)
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = matvec(V[j])
            for i in range(j + 1):  # modified Gram-Schmidt
                H[i, j] = np.dot(V[i], w)
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):  # apply earlier rotations to the new column
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            k = j + 1
            hist.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or iters >= max_iter:
                break
        # least squares: back substitution on the k x k upper triangle
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + V[:k].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        rel = beta / bnorm
    return x, dict(iters=iters, converged=rel <= tol, history=hist, rel_residual=rel)
