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


# --------------------------------------------------------------------------
# Learned approximate-cardinal preconditioner: plain references.
# --------------------------------------------------------------------------
def knn(X, k):
    """k nearest centres of every centre (itself included): ascending squared distance
    sum_t (x_t - y_t)^2 (FP64, dimension order 0..d-1), ties broken by original index."""
    X = np.asarray(X, dtype=np.float64)
    n = len(X)
    out = np.empty((n, k), dtype=np.int64)
    idx = np.arange(n)
    for i in range(n):
        d2 = np.zeros(n)
        for t in range(X.shape[1]):
            q = X[:, t] - X[i, t]
            d2 = d2 + q * q
        order = np.lexsort((idx, d2))
        out[i] = order[:k]
    return out


def features(X, nbr, eps):
    """eps * (x_j - x_i) for the neighbours j of i in distance order, flattened (k*d)."""
    X = np.asarray(X, dtype=np.float64)
    return (eps * (X[nbr] - X[:, None, :])).reshape(len(X), -1)


def cardinal(X, nbr_rows, kernel, eps, delta_rel):
    """Local cardinal coefficients c = (A_S + delta I)^-1 e_1 on each neighbour set S
    (first entry = the centre itself), delta = delta_rel * ||A_S||_F."""
    from oracle import phi
    X = np.asarray(X, dtype=np.float64)
    out = np.empty(nbr_rows.shape, dtype=np.float64)
    k = nbr_rows.shape[1]
    for i, S in enumerate(nbr_rows):
        P = X[S]
        A = phi(kernel, eps, np.linalg.norm(P[:, None, :] - P[None, :, :], axis=2))
        A = A + delta_rel * np.linalg.norm(A) * np.eye(k)
        e = np.zeros(k)
        e[0] = 1.0
        out[i] = np.linalg.solve(A, e)
    return out


def mlp_init(sizes, seed):
    """He-normal weights W[l] (out x in) and zero biases."""
    rng = np.random.default_rng(seed)
    W, b = [], []
    for a, c in zip(sizes[:-1], sizes[1:]):
        W.append(rng.standard_normal((c, a)) * np.sqrt(2.0 / a))
        b.append(np.zeros(c))
    return W, b


def bf16_round(a):
    """Round to the nearest BF16 value (8 significant bits, ties to even), returned as FP64:
    the operand precision of a BF16 tensor-core product."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def mlp_forward(W, b, X, q=None):
    """h_0 = X; z_l = q(h_{l-1}) q(W_l)^T + b_l; h_l = relu(z_l) on hidden layers; y = z_last.
    q rounds the operands of each product (identity by default; bf16_round gives the operand
    precision of a BF16 network, with the sums still in FP64)."""
    q = q or (lambda a: a)
    h = [np.asarray(X, dtype=np.float64)]
    z = []
    for l in range(len(W)):
        zl = q(h[-1]) @ q(W[l]).T + b[l]
        z.append(zl)
        h.append(np.maximum(zl, 0.0) if l < len(W) - 1 else zl)
    return h[-1], (h, z)


def mse_loss(Y, T):
    return float(np.mean((Y - T) ** 2))


def mlp_backward(W, b, cache, Y, T, q=None):
    """Gradients of mse_loss(Y, T) w.r.t. every W_l and b_l (chain rule, FP64 sums; q rounds
    the operands of each product as in mlp_forward)."""
    q = q or (lambda a: a)
    h, z = cache
    g = 2.0 * (Y - T) / Y.size
    gW, gb = [None] * len(W), [None] * len(W)
    for l in range(len(W) - 1, -1, -1):
        if l < len(W) - 1:
            g = g * (z[l] > 0)
        gW[l] = q(g).T @ q(h[l])
        gb[l] = g.sum(axis=0)
        g = q(g) @ q(W[l])
    return gW, gb


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of parameters p in place; t counts from 1."""
    m[:] = b1 * m + (1 - b1) * g
    v[:] = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    p[:] = p - lr * mh / (np.sqrt(vh) + eps)
