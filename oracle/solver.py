"""Plain FP64 reference algorithms for the interpolation solve and the learned
preconditioner.  TEST INFRASTRUCTURE ONLY (see oracle/__init__.py)."""
from __future__ import annotations

import numpy as np


def gmres(matvec, b, x0=None, m=50, tol=1e-8, maxit=1000):
    """Restarted GMRES(m) for A x = b (Saad & Schultz): Arnoldi with classical
    Gram-Schmidt applied twice, Givens rotations on the Hessenberg matrix,
    restart from the true residual.  Stops when ||b - A x|| <= tol ||b||.
    Returns (x, iterations, relative residual history at restarts)."""
    b = np.asarray(b, dtype=np.float64)
    n = len(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0, [0.0]
    it = 0
    r = b - matvec(x)
    beta = np.linalg.norm(r)
    hist = [beta / nb]
    while beta > tol * nb and it < maxit:
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j = 0
        while j < m and it < maxit:
            w = matvec(V[j])
            h = np.zeros(j + 2)
            for _ in range(2):                       # classical Gram-Schmidt, twice
                c = V[:j + 1] @ w
                w = w - V[:j + 1].T @ c
                h[:j + 1] += c
            h[j + 1] = np.linalg.norm(w)
            for k in range(j):                       # previous rotations
                h[k], h[k + 1] = cs[k] * h[k] + sn[k] * h[k + 1], -sn[k] * h[k] + cs[k] * h[k + 1]
            den = np.hypot(h[j], h[j + 1])
            cs[j], sn[j] = (h[j] / den, h[j + 1] / den) if den > 0 else (1.0, 0.0)
            hn = h[j + 1]
            h[j], h[j + 1] = den, 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            H[:j + 1, j] = h[:j + 1]
            it += 1
            j += 1
            if hn > 0:
                V[j] = w / hn
            if abs(g[j]) <= tol * nb or hn == 0:
                break
        y = np.linalg.solve(np.triu(H[:j, :j]), g[:j])
        x = x + V[:j].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        hist.append(beta / nb)
    return x, it, hist
