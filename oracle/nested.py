"""FP64 oracle of the MLFMM on scale-invariant (nested) frequency grids.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may use it.

The paper's MLFMM (Sec. 4.1, "Upsweep", "Coupling", "Downsweep", and
Sec. 4.1.1 "Interpolation and Anterpolation") keeps the same number of nodes M
on every level and scales the frequency grid with the box: the grid of level
l-1 is the grid of level l halved, xi_{l-1} = xi_l / 2 (the scaling property of
the Fourier transform).  The expansions of a parent are therefore needed at
frequencies where the children have no samples, and the paper obtains them by
polynomial (Lagrange) interpolation in xi:

  M2M, Eq. (43):  V_p(xi_{l-1}) = sum_c e^{-i xi_{l-1}.(c_c - c_p)} [P V_c](xi_{l-1})
  M2L, Eq. (45):  L_a(xi_l)   += omega_l C_l(xi_l) e^{i xi_l.(c_a - c_b)} V_b(xi_l),  b in IL_l(a)
  L2L, Eqs. (47)-(48): L_c(xi_l) += [P^T (e^{i xi_{l-1}.(c_c - c_p)} L_p)](xi_l)
  P2M / L2P at the leaves on the leaf grid xi_D.

Readings fixed here (each is also listed in the design notes):

* Grid of level l: the shared-grid construction with period
  L_l = L * 2^(2-l) (level 2 keeps the period L of the shared grid), so
  dxi_l = 2 pi / L_l and xi_{l-1} = xi_l / 2 exactly; M nodes per dimension on
  every level.
* Coefficients of level l: C_l from lattice samples of the kernel exactly as on
  the shared grid, with period L_l and the taper's flat radius
  R_in,l = side * 2^(2-l) (4 boxes of level l, the largest far offset
  component of IL_l).
* Interpolation P: one dimension at a time (tensor product).  The standard
  Lagrange basis l_k(t) = prod_{m != k} (t - t_m) / (t_k - t_m) (the printed
  formula of Sec. 4.1.1 has its indices swapped) on K consecutive child nodes
  around the target: in node units the target k' of the parent grid sits at
  k'/2 on the child grid and uses the child nodes floor(k'/2) - K/2 + 1 ..
  floor(k'/2) + K/2.  Even k' fall on a child node (the weight is exactly 1).
  The node set of the paper's error table (K equispaced nodes on [-pi, pi],
  targets xi/2) reproduces that table with this basis.
* Anterpolation is the transpose P^T of the same matrix (Eq. (51)); omega is
  applied once per far pair, in M2L (as on the shared grid).
* Operator order as printed: each child is interpolated first and then
  translated (Eq. (43)); the parent's local expansion is translated first and
  then anterpolated (Eq. (47)).
"""
from __future__ import annotations

import numpy as np

from . import box_centres, coeffs_sampled, freq_grid, l2p, m2l, p2m, p2p


# --------------------------------------------------------------------------
# Lagrange interpolation in xi (Sec. 4.1.1)
# --------------------------------------------------------------------------
def lagrange_basis(nodes, t):
    """l_k(t) = prod_{m != k} (t - nodes_m) / (nodes_k - nodes_m); returns [len(t)][K]."""
    nodes = np.asarray(nodes, dtype=np.float64)
    t = np.atleast_1d(np.asarray(t, dtype=np.float64))
    K = len(nodes)
    out = np.ones((len(t), K))
    for k in range(K):
        for m in range(K):
            if m != k:
                out[:, k] *= (t - nodes[m]) / (nodes[k] - nodes[m])
    return out


def lagrange_halfwave_error(K: int, a: float = 1.0, n_eval: int = 38):
    """Sup-norm error of interpolating e^{i (xi/2) x} from K equispaced nodes
    xi_k on [-pi, pi] (end points included), over xi in [-pi, pi] and x in
    [-a, a], both sampled on n_eval equispaced points (the setting of the
    paper's table "Lagrange interpolation error", Sec. 4.1.1)."""
    nodes = np.linspace(-np.pi, np.pi, K)
    xi = np.linspace(-np.pi, np.pi, n_eval)
    x = np.linspace(-a, a, n_eval)
    P = lagrange_basis(nodes, xi / 2.0)
    exact = np.exp(1j * np.outer(xi / 2.0, x))
    approx = P @ np.exp(1j * np.outer(nodes, x))
    return float(np.max(np.abs(exact - approx)))


def stencil_start(k: int, K: int) -> int:
    """First child node (index k = -M/2..M/2 units) of parent node k's stencil."""
    return (k // 2) - K // 2 + 1


def interp_matrix(M: int, K: int):
    """P[k', j']: weight of child node j on parent node k' (primes: +M/2), both
    on k = -M/2..M/2.  Row k' holds the Lagrange basis of the K child nodes
    around k/2, evaluated at k/2 (node units; the basis is scale free)."""
    if K % 2 or K < 2 or M < 2 * K:
        raise ValueError("K must be even, >= 2, and M >= 2K")
    n1 = M + 1
    P = np.zeros((n1, n1))
    for kp in range(n1):
        k = kp - M // 2
        j0 = stencil_start(k, K)
        nodes = np.arange(j0, j0 + K, dtype=np.float64)
        P[kp, j0 + M // 2:j0 + M // 2 + K] = lagrange_basis(nodes, k / 2.0)[0]
    return P


# --------------------------------------------------------------------------
# Level grids and coefficients
# --------------------------------------------------------------------------
def level_period(L: float, l: int) -> float:
    """L_l = L * 2^(2-l)."""
    return L * 2.0 ** (2 - l)


def coeffs_levels(kernel: int, eps: float, d: int, M: int, L: float, alpha: float, side: float, D: int):
    """{l: omega_l C_l} for l = 2..D (full grid, dimension 0 fastest)."""
    return {l: coeffs_sampled(kernel, eps, d, M, level_period(L, l), alpha, side * 2.0 ** (2 - l))
            for l in range(2, D + 1)}


def _as_grid(A, d: int, M: int):
    """[nbox][(M+1)^d] (dimension 0 fastest) -> [nbox][n1]*d with axis 1 + (d-1-t) <-> dimension t."""
    return A.reshape((A.shape[0],) + (M + 1,) * d)


def _phase(xi, delta):
    """e^{i xi_k . delta} on the full grid, shaped [n1]*d with axis d-1-t <-> dimension t; delta [d]."""
    d = len(delta)
    ph = np.ones(())
    for t in range(d - 1, -1, -1):
        ph = np.multiply.outer(ph, np.exp(1j * xi * delta[t]))
    return ph


def _apply_axes(A, P, transpose: bool):
    """Apply P (or P^T) along every grid axis of A [nbox][n1]*d."""
    for ax in range(1, A.ndim):
        A = np.moveaxis(np.tensordot(A, P, axes=([ax], [0 if transpose else 1])), -1, ax)
    return A


def m2m(T, Vc, child_level: int, M: int, L: float, K: int):
    """Eq. (43): parents at level child_level-1 from their children."""
    d = T["d"]
    lp = child_level - 1
    xi_p, _ = freq_grid(M, level_period(L, lp))
    P = interp_matrix(M, K)
    ch, par = T["levels"][child_level], T["levels"][lp]
    cc = box_centres(ch["key"], d, child_level, T["lo"], T["side"])
    pc = box_centres(par["key"], d, lp, T["lo"], T["side"])
    W = _apply_axes(_as_grid(Vc, d, M), P, transpose=False)
    Vp = np.zeros((len(par["key"]),) + (M + 1,) * d, dtype=np.complex128)
    for c in range(len(ch["key"])):
        p = ch["parent"][c]
        Vp[p] += _phase(xi_p, -(cc[c] - pc[p])) * W[c]
    return Vp.reshape(len(par["key"]), -1)


def l2l(T, Lp, Lc, child_level: int, M: int, L: float, K: int):
    """Eqs. (47)-(48): Lc += P^T (e^{i xi_{l-1}.(c_c - c_p)} L_p) for every child."""
    d = T["d"]
    lp = child_level - 1
    xi_p, _ = freq_grid(M, level_period(L, lp))
    P = interp_matrix(M, K)
    ch, par = T["levels"][child_level], T["levels"][lp]
    cc = box_centres(ch["key"], d, child_level, T["lo"], T["side"])
    pc = box_centres(par["key"], d, lp, T["lo"], T["side"])
    G = _as_grid(Lp, d, M)
    S = np.empty((len(ch["key"]),) + (M + 1,) * d, dtype=np.complex128)
    for c in range(len(ch["key"])):
        p = ch["parent"][c]
        S[c] = _phase(xi_p, cc[c] - pc[p]) * G[p]
    Lc += _apply_axes(S, P, transpose=True).reshape(len(ch["key"]), -1)


def fmm(T, lam, kernel: int, eps: float, wcs, M: int, L: float, K: int, return_parts: bool = False):
    """The MLFMM product of Sec. 4.1 on nested grids, FP64, in the paper's order:
    P2M on the leaf grid -> M2M (Eq. (43)) to level 2 -> M2L on every level
    2..D with that level's grid and coefficients (Eq. (45)) -> L2L (Eq. (48))
    -> L2P on the leaf grid (Eq. (46)); near field as Eq. (38).
    wcs = coeffs_levels(...).  lam and the result are in the original order."""
    D = T["D"]
    lam = np.asarray(lam, dtype=np.float64)
    ls = lam[T["perm"]]
    u_near = p2p(T, ls, kernel, eps)
    u_far = np.zeros(T["N"])
    if D >= 2:
        V = {D: p2m(T, ls, M, level_period(L, D))}
        for l in range(D, 2, -1):
            V[l - 1] = m2m(T, V[l], l, M, L, K)
        Lx = {l: np.zeros_like(V[l]) for l in range(2, D + 1)}
        for l in range(2, D + 1):
            m2l(T, V[l], Lx[l], l, wcs[l], M, level_period(L, l))
        for l in range(3, D + 1):
            l2l(T, Lx[l - 1], Lx[l], l, M, L, K)
        l2p(T, Lx[D], M, level_period(L, D), u_far)
    us = u_near + u_far
    u = np.empty_like(us)
    u[T["perm"]] = us
    if return_parts:
        un = np.empty_like(us)
        un[T["perm"]] = u_near
        return u, un
    return u


# --------------------------------------------------------------------------
# Pair-by-pair restatement (tests only): what the nested FMM computes for one
# far pair, built from one-dimensional phase chains instead of box expansions.
# --------------------------------------------------------------------------
def _chain(x, c_leaf, centres, M, L, K, l_top, D, sign):
    """One dimension: the approximation on level l_top's grid of
    e^{sign i xi (x - c_{l_top})}, obtained from the exact leaf phases by
    interpolating and translating level by level (centres[l] = box centre at l)."""
    P = interp_matrix(M, K)
    xi_D, _ = freq_grid(M, level_period(L, D))
    v = np.exp(sign * 1j * xi_D * (x - c_leaf))
    for l in range(D, l_top, -1):
        xi_p, _ = freq_grid(M, level_period(L, l - 1))
        v = np.exp(sign * 1j * xi_p * (centres[l] - centres[l - 1])) * (P @ v)
    return v


def fmm_pairwise(X, lam, lo, side: float, D: int, kernel: int, eps: float, wcs, M: int, L: float,
                 K: int):
    """u_i = sum_{near} Phi lambda_j + sum_{far} Re sum_{xi_l} omega_l C_l(xi_l)
    A_i(xi_l) e^{i xi_l.(c_a - c_b)} B_j(xi_l) lambda_j, where l is the level at
    which the boxes of i and j are separated (not adjacent, parents adjacent),
    and A_i, B_j are the per-dimension chains of interpolated phases.  Pairs are
    classified from the box coordinates directly.  O(N^2 M^d); tiny N only."""
    from . import phi
    X = np.asarray(X, dtype=np.float64)
    N, d = X.shape
    lo = np.asarray(lo, dtype=np.float64)
    kD = np.clip(np.floor(((X - lo) / side) * 2 ** D).astype(np.int64), 0, 2 ** D - 1)

    def centre(kl, l):
        return lo + (kl + 0.5) * (side / 2 ** l)

    # chains per point, per level, per dimension: A (target, +) and B (source, -)
    A, B = {}, {}
    for i in range(N):
        cents = {l: centre(kD[i] >> (D - l), l) for l in range(2, D + 1)}
        for l in range(2, D + 1):
            A[i, l] = [_chain(X[i, t], cents[D][t], {q: cents[q][t] for q in cents}, M, L, K, l, D, +1)
                       for t in range(d)]
            B[i, l] = [_chain(X[i, t], cents[D][t], {q: cents[q][t] for q in cents}, M, L, K, l, D, -1)
                       for t in range(d)]
    u = np.zeros(N)
    for i in range(N):
        for j in range(N):
            if np.max(np.abs(kD[i] - kD[j])) <= 1:
                u[i] += phi(kernel, eps, np.linalg.norm(X[i] - X[j])) * lam[j]
                continue
            l = next(q for q in range(2, D + 1)
                     if np.max(np.abs((kD[i] >> (D - q)) - (kD[j] >> (D - q)))) >= 2)
            xi_l, _ = freq_grid(M, level_period(L, l))
            dc = centre(kD[i] >> (D - l), l) - centre(kD[j] >> (D - l), l)
            prod = np.ones(())
            for t in range(d - 1, -1, -1):
                prod = np.multiply.outer(prod, A[i, l][t] * np.exp(1j * xi_l * dc[t]) * B[j, l][t])
            u[i] += np.real(np.sum(wcs[l] * prod.ravel())) * lam[j]
    return u


def kernel_levels_error(kernel: int, eps: float, d: int, M: int, L: float, wcs, side: float, D: int,
                        n: int = 2000, seed: int = 0):
    """Largest |K_l(r) - Phi(r)| over sampled far offsets of each level l
    (components |r_t| <= 4 side_l, at least one >= side_l)."""
    from . import kernel_K, phi
    rng = np.random.default_rng(seed)
    worst = 0.0
    for l in range(2, D + 1):
        s = side * 2.0 ** -l
        r = rng.uniform(-4 * s, 4 * s, (n, d))
        big = np.max(np.abs(r), axis=1) >= s
        r = r[big]
        err = np.abs(kernel_K(wcs[l], d, M, level_period(L, l), r) - phi(kernel, eps, np.linalg.norm(r, axis=1)))
        worst = max(worst, float(err.max()))
    return worst

