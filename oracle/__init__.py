"""Plain FP64 CPU oracle for the band-limited FMM of Zhao & Stoll (arXiv 1606.07652).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code,
header, table or helper with the CUDA library, and the CUDA library never
imports it.

Layout of the oracle:

* this module (numpy): the frequency grid, the coefficient tables C(xi), the
  Morton tree and its lists, and the FMM driver that calls the passes in the
  paper's order;
* ``rbf_oracle.c`` (plain C99 + OpenMP over independent outputs): the heavy
  loops -- near field, P2M, M2M, M2L, L2L, L2P, the direct sum and the far
  kernel K;
* ``solver.py``: GMRES, the local cardinal solves, k-nearest neighbours and
  the MLP of the learned preconditioner.

Readings of the paper that this oracle fixes (each is also listed in the
project's design notes):

* Grid, Sec. 3.2 (the choices after Eq. (P2M)): dxi = 2 pi / L, h = L / M,
  sigma = M dxi / 2 = pi / h.  Nodes xi_k = k dxi, k = -M/2 .. M/2 in every
  dimension, with the symmetric half weight dxi/2 at k = +-M/2 and dxi
  elsewhere (the "symmetric +-sigma half-weight" form of the paper's
  left-endpoint rule; it makes K real and even).
* Coefficients, Eq. (M2Loperator) generalised from unit spacing to spacing h
  and to d dimensions with the (2 pi)^-d of Eq. (29):
      C(xi) = (2 pi)^-d h^d sum_q f(q) e^{-i xi . q h},  q in {-M/2..M/2-1}^d,
  where f(q) = sum_{n in {-1,0,1}^d} Phi(qh + nL) prod_t w(qh_t + n_t L) is the
  sampled kernel periodised with period L and, for slowly decaying kernels,
  tapered by the window w(t) = erfc(alpha (2(|t|-R_in)/(L-2 R_in) - 1)) / 2.
* Closed-form coefficients for the Gaussian (validation only):
  C(xi) = (2 pi)^-d Phi_hat(xi), Phi_hat(xi) = (pi/eps^2)^{d/2} e^{-|xi|^2/(4 eps^2)}
  (Fourier transform in the convention of Eq. (5)).
* Far kernel, Eq. (35): K(r) = sum_xi omega(xi) C(xi) e^{i xi . r} (real).
* Tree: level-uniform 2^d-tree over the root cube [lo, lo+side]^d; integer box
  coordinate k_t = min(max(floor(((x_t - lo_t)/side) * 2^D), 0), 2^D - 1);
  Morton key with dimension 0 in the least significant bit; stable sort by
  (key, original index).  Near list N_a: leaves at Chebyshev index distance
  <= 1 (self included), Eq. (38).  Interaction list IL_l(a): level-l boxes
  whose parent is within Chebyshev distance 1 of a's parent and that are at
  distance >= 2 from a (Sec. 4.1 coupling on every level 2..D).
* One shared frequency grid on all levels (interpolation operator P = I in
  Eqs. (43) and (48)); omega is applied exactly once per far pair, in M2L.
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess

import numpy as np

GAUSSIAN = 0
IMQ = 1
MQ = 2
WENDLAND = 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "rbf_oracle.c")
_lib = None


def build(force: bool = False) -> str:
    """Compile rbf_oracle.c into oracle/_build/liboracle.so (gcc, -fopenmp)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.orc_phi.restype = ctypes.c_double
        _lib.orc_phi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
        _lib.orc_num_threads.restype = ctypes.c_int
    return _lib


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's OpenMP loops from now on (for timing on one core)."""
    lib().orc_set_num_threads(ctypes.c_int(int(n)))


def _p(a):
    # data_as keeps a reference to the array inside the pointer object, so a
    # temporary (a converted copy built in the argument list) stays alive for
    # the duration of the call
    return a.ctypes.data_as(ctypes.c_void_p)


_I = ctypes.c_int
_L = ctypes.c_int64
_D = ctypes.c_double


# --------------------------------------------------------------------------
# Kernels: Tables "Global functions" and "Compactly supported functions"
# (Sec. 2.2), shape-parameter form.
# --------------------------------------------------------------------------
def phi(kernel: int, eps: float, r):
    """Phi(r) = exp(-(eps r)^2) (Gaussian), 1/sqrt(1+(eps r)^2) (IMQ),
    sqrt(1+(eps r)^2) (MQ) or (1 - eps r)_+^3 (3 eps r + 1) (Wendland Phi_{2,1})."""
    er = eps * np.asarray(r, dtype=np.float64)
    if kernel == GAUSSIAN:
        return np.exp(-er * er)
    if kernel == MQ:
        return np.sqrt(1.0 + er * er)
    if kernel == WENDLAND:
        t = np.where(er < 1.0, 1.0 - er, 0.0)
        return t * t * t * (3.0 * er + 1.0)
    return 1.0 / np.sqrt(1.0 + er * er)


# --------------------------------------------------------------------------
# Frequency grid and coefficients, Sec. 3.2 (Eqs. quadrature, M2Loperator,
# 28, 29) under the readings stated in the module docstring.
# --------------------------------------------------------------------------
def freq_grid(M: int, L: float):
    """1-D nodes xi_k = k*2pi/L, k=-M/2..M/2, and their weights (half at the ends)."""
    if M % 2 or M < 2:
        raise ValueError("M must be even and >= 2")
    dxi = 2.0 * np.pi / L
    k = np.arange(-M // 2, M // 2 + 1)
    xi = k * dxi
    w = np.full(M + 1, dxi)
    w[0] *= 0.5
    w[-1] *= 0.5
    return xi, w


def window(t, L: float, R_in: float, alpha: float):
    """Taper w(t) = erfc(alpha (2(|t|-R_in)/(L-2R_in) - 1)) / 2; 1 when alpha == 0."""
    from scipy.special import erfc
    t = np.abs(np.asarray(t, dtype=np.float64))
    if alpha == 0.0:
        return np.ones_like(t)
    return 0.5 * erfc(alpha * (2.0 * (t - R_in) / (L - 2.0 * R_in) - 1.0))


def lattice_samples(kernel: int, eps: float, d: int, M: int, L: float, alpha: float, R_in: float):
    """f(q), q in {-M/2..M/2-1}^d: Phi * window at qh, summed over the 3^d images qh + nL.

    Returned as an array of shape (M,)*d indexed by q + M/2, axis a <-> dimension a."""
    h = L / M
    q = np.arange(-M // 2, M // 2) * h
    f = np.zeros((M,) * d)
    grids = np.meshgrid(*([q] * d), indexing="ij")
    for n in itertools.product((-1, 0, 1), repeat=d):
        comps = [grids[t] + n[t] * L for t in range(d)]
        r = np.sqrt(sum(c * c for c in comps))
        wprod = np.ones_like(r)
        for c in comps:
            wprod = wprod * window(c, L, R_in, alpha)
        f += phi(kernel, eps, r) * wprod
    return f


def coeffs_sampled(kernel: int, eps: float, d: int, M: int, L: float, alpha: float, R_in: float):
    """omega*C on the full symmetric grid, flattened with dimension 0 fastest.

    C(xi_k) = (2pi)^-d h^d sum_q f(q) e^{-i xi_k . qh}  (Eq. (M2Loperator), spacing h),
    evaluated with numpy's FFT (e^{-i xi_k q h} = e^{-2 pi i k q / M})."""
    h = L / M
    f = lattice_samples(kernel, eps, d, M, L, alpha, R_in)
    D = np.fft.fftn(np.fft.ifftshift(f))          # D[k mod M] = sum_q f(q) e^{-2pi i k.q/M}
    if np.max(np.abs(D.imag)) > 1e-9 * max(1.0, np.max(np.abs(D.real))):
        raise AssertionError("sampled kernel is not even")
    idx = np.arange(-M // 2, M // 2 + 1) % M
    Cfull = D.real[np.ix_(*([idx] * d))] * (h ** d) / (2.0 * np.pi) ** d
    return _omega_times(Cfull, M, L, d)


def coeffs_closed_gaussian(eps: float, d: int, M: int, L: float):
    """omega*C with C = (2pi)^-d Phi_hat(xi), Phi_hat = (pi/eps^2)^{d/2} e^{-|xi|^2/(4eps^2)}."""
    xi, _ = freq_grid(M, L)
    g = np.meshgrid(*([xi] * d), indexing="ij")
    xi2 = sum(c * c for c in g)
    C = (np.pi / eps ** 2) ** (d / 2.0) * np.exp(-xi2 / (4.0 * eps * eps)) / (2.0 * np.pi) ** d
    return _omega_times(C, M, L, d)


def _omega_times(C, M, L, d):
    _, w = freq_grid(M, L)
    W = np.ones(())
    for _t in range(d):
        W = np.multiply.outer(W, w)
    wc = W * C                                   # axis a <-> dimension a
    # flatten with dimension 0 fastest: C-order flattening makes the LAST axis
    # fastest, so reverse the axes first.
    return np.ascontiguousarray(np.transpose(wc, axes=tuple(range(d - 1, -1, -1)))).ravel()


def kernel_K(omegaC, d: int, M: int, L: float, r):
    """Eq. (35): K(r) = Re sum_xi omega C(xi) e^{i xi.r}; r is (n, d)."""
    xi, _ = freq_grid(M, L)
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1, d))
    out = np.zeros(r.shape[0])
    lib().orc_kernel_K(_I(d), _I(M), _p(xi), _p(np.ascontiguousarray(omegaC, dtype=np.float64)),
                       _L(r.shape[0]), _p(r), _p(out))
    return out


# --------------------------------------------------------------------------
# Tree and lists (Sec. 1 step list "hierarchical tree"; N_a, G_b of Eq. (38);
# interaction lists of the MLFMM coupling, Sec. 4.1).
# --------------------------------------------------------------------------
def morton_encode(k, d: int, D: int):
    """Interleave integer coordinates k[..., d]: bit b of dim t -> key bit b*d + t."""
    k = np.asarray(k, dtype=np.uint64)
    key = np.zeros(k.shape[:-1], dtype=np.uint64)
    for b in range(D):
        for t in range(d):
            key |= ((k[..., t] >> np.uint64(b)) & np.uint64(1)) << np.uint64(b * d + t)
    return key


def morton_decode(key, d: int, l: int):
    key = np.asarray(key, dtype=np.uint64)
    k = np.zeros(key.shape + (d,), dtype=np.int64)
    for b in range(l):
        for t in range(d):
            k[..., t] |= (((key >> np.uint64(b * d + t)) & np.uint64(1)).astype(np.int64)) << b
    return k


def box_coords(X, lo, side: float, D: int):
    """k_t = min(max(floor(((x_t - lo_t)/side) * 2^D), 0), 2^D-1), in FP64."""
    X = np.asarray(X, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.float64)
    k = np.floor(((X - lo) / side) * float(2 ** D)).astype(np.int64)
    return np.clip(k, 0, 2 ** D - 1)


def box_centres(keys, d: int, l: int, lo, side: float):
    k = morton_decode(keys, d, l).astype(np.float64)
    return np.asarray(lo, dtype=np.float64) + (k + 0.5) * (side / 2 ** l)


def _csr(pairs_a, pairs_b, n):
    order = np.lexsort((pairs_b, pairs_a))
    a, b = pairs_a[order], pairs_b[order]
    off = np.zeros(n + 1, dtype=np.int64)
    np.add.at(off, a + 1, 1)
    return np.cumsum(off), b.astype(np.int64)


def _lookup(keys_sorted, q):
    pos = np.searchsorted(keys_sorted, q)
    pos_c = np.minimum(pos, len(keys_sorted) - 1)
    ok = (pos < len(keys_sorted)) & (keys_sorted[pos_c] == q)
    return ok, pos_c


def tree(X, lo, side: float, D: int):
    """Morton tree of the centres X (N, d).  Returns a dict of numpy arrays:

    perm      sorted position -> original index (stable by (key, index))
    keys      Morton keys of the sorted points (uint64, level D)
    xs        sorted points (N, d)
    leaf_key  Morton keys of the non-empty leaves, ascending
    leaf_off  point offsets of the non-empty leaves (nleaf+1)
    near_off, near_idx   CSR near lists over compact leaf ids
    levels[l] for l = 0..D: dict(key, parent (compact id at l-1), child_off
              (children at l+1), il_off, il_idx (levels >= 2))
    """
    X = np.asarray(X, dtype=np.float64)
    N, d = X.shape
    lo = np.asarray(lo, dtype=np.float64).reshape(d)
    k = box_coords(X, lo, side, D)
    key = morton_encode(k, d, D)
    perm = np.argsort(key, kind="stable")
    ks = key[perm]
    leaf_key, first = np.unique(ks, return_index=True)
    leaf_off = np.append(first, N).astype(np.int64)
    nleaf = len(leaf_key)

    # near lists: leaves at Chebyshev distance <= 1, self included
    kc = morton_decode(leaf_key, d, D)
    A, B = [], []
    for delta in itertools.product((-1, 0, 1), repeat=d):
        nb = kc + np.array(delta)
        inside = np.all((nb >= 0) & (nb < 2 ** D), axis=1)
        ok, pos = _lookup(leaf_key, morton_encode(np.clip(nb, 0, 2 ** D - 1), d, D))
        sel = inside & ok
        A.append(np.nonzero(sel)[0])
        B.append(pos[sel])
    near_off, near_idx = _csr(np.concatenate(A), np.concatenate(B), nleaf)

    levels = {}
    for l in range(D, -1, -1):
        lk = np.unique(leaf_key >> np.uint64(d * (D - l)))
        levels[l] = {"key": lk}
    for l in range(1, D + 1):
        parent_keys = levels[l]["key"] >> np.uint64(d)
        levels[l]["parent"] = np.searchsorted(levels[l - 1]["key"], parent_keys).astype(np.int64)
        off = np.zeros(len(levels[l - 1]["key"]) + 1, dtype=np.int64)
        np.add.at(off, levels[l]["parent"] + 1, 1)
        levels[l - 1]["child_off"] = np.cumsum(off)
    for l in range(2, D + 1):
        bk = levels[l]["key"]
        bc = morton_decode(bk, d, l)
        pc = bc >> 1
        A, B = [], []
        for dp in itertools.product((-1, 0, 1), repeat=d):
            for ch in itertools.product((0, 1), repeat=d):
                cand = 2 * (pc + np.array(dp)) + np.array(ch)
                inside = np.all((cand >= 0) & (cand < 2 ** l), axis=1)
                well_sep = np.max(np.abs(cand - bc), axis=1) >= 2
                ok, pos = _lookup(bk, morton_encode(np.clip(cand, 0, 2 ** l - 1), d, l))
                sel = inside & well_sep & ok
                A.append(np.nonzero(sel)[0])
                B.append(pos[sel])
        levels[l]["il_off"], levels[l]["il_idx"] = _csr(np.concatenate(A), np.concatenate(B), len(bk))
    return {"N": N, "d": d, "D": D, "lo": lo, "side": float(side), "perm": perm, "keys": ks,
            "xs": np.ascontiguousarray(X[perm]), "leaf_key": leaf_key, "leaf_off": leaf_off,
            "near_off": near_off, "near_idx": near_idx, "levels": levels}


# --------------------------------------------------------------------------
# The matrix-vector product, Eq. (1) and Eq. (38)/(54).
# --------------------------------------------------------------------------
def direct(X, lam, kernel: int, eps: float, targets=None):
    """Eq. (1): u_i = sum_j lambda_j Phi(x_i - x_j) for the given targets (all by default)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    N, d = X.shape
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    t = np.arange(N, dtype=np.int64) if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    u = np.zeros(len(t))
    lib().orc_direct(_L(N), _I(d), _p(X), _p(lam), _I(kernel), _D(eps), _L(len(t)), _p(t), _p(u))
    return u


def p2p(T, lam_sorted, kernel: int, eps: float):
    """Near field of Eq. (38) on sorted points; returns u_near in sorted order."""
    u = np.zeros(T["N"])
    lam_sorted = np.ascontiguousarray(lam_sorted, dtype=np.float64)
    lib().orc_p2p(_I(T["d"]), _L(len(T["leaf_key"])), _p(T["leaf_off"]), _p(T["near_off"]),
                  _p(T["near_idx"]), _p(T["xs"]), _p(lam_sorted), _I(kernel), _D(eps), _p(u))
    return u


def n_modes(d: int, M: int) -> int:
    return (M + 1) ** d


def p2m(T, lam_sorted, M: int, L: float):
    d, D = T["d"], T["D"]
    xi, _ = freq_grid(M, L)
    nb = len(T["leaf_key"])
    V = np.zeros((nb, n_modes(d, M)), dtype=np.complex128)
    lib().orc_p2m(_I(d), _I(M), _p(xi), _L(nb), _p(T["leaf_key"]), _I(D), _p(T["lo"]),
                  _D(T["side"]), _p(T["leaf_off"]), _p(T["xs"]),
                  _p(np.ascontiguousarray(lam_sorted, dtype=np.float64)), _p(V))
    return V


def m2m(T, Vc, child_level: int, M: int, L: float):
    d = T["d"]
    xi, _ = freq_grid(M, L)
    par = T["levels"][child_level - 1]
    Vp = np.zeros((len(par["key"]), n_modes(d, M)), dtype=np.complex128)
    lib().orc_m2m(_I(d), _I(M), _p(xi), _I(child_level), _p(T["lo"]), _D(T["side"]),
                  _L(len(par["key"])), _p(par["key"]), _p(par["child_off"]),
                  _p(T["levels"][child_level]["key"]), _p(np.ascontiguousarray(Vc)), _p(Vp))
    return Vp


def m2l(T, V, Lx, level: int, omegaC, M: int, L: float):
    d = T["d"]
    xi, _ = freq_grid(M, L)
    lv = T["levels"][level]
    lib().orc_m2l(_I(d), _I(M), _p(xi), _p(np.ascontiguousarray(omegaC)), _I(level), _p(T["lo"]),
                  _D(T["side"]), _L(len(lv["key"])), _p(lv["key"]), _p(lv["il_off"]),
                  _p(lv["il_idx"]), _p(np.ascontiguousarray(V)), _p(Lx))


def l2l(T, Lp, Lc, child_level: int, M: int, L: float):
    d = T["d"]
    xi, _ = freq_grid(M, L)
    ch = T["levels"][child_level]
    lib().orc_l2l(_I(d), _I(M), _p(xi), _I(child_level), _p(T["lo"]), _D(T["side"]),
                  _L(len(ch["key"])), _p(ch["key"]), _p(ch["parent"]),
                  _p(T["levels"][child_level - 1]["key"]), _p(np.ascontiguousarray(Lp)), _p(Lc))


def l2p(T, Lleaf, M: int, L: float, u):
    d, D = T["d"], T["D"]
    xi, _ = freq_grid(M, L)
    lib().orc_l2p(_I(d), _I(M), _p(xi), _L(len(T["leaf_key"])), _p(T["leaf_key"]), _I(D),
                  _p(T["lo"]), _D(T["side"]), _p(T["leaf_off"]), _p(T["xs"]),
                  _p(np.ascontiguousarray(Lleaf)), _p(u))


def fmm(T, lam, kernel: int, eps: float, omegaC, M: int, L: float, return_parts: bool = False):
    """The multilevel FMM matvec of Sec. 4 in the paper's order, FP64.

    u = A_near lambda (Eq. (38) near field) + U K V lambda (Eq. (54)):
      P2M at the leaves -> M2M upsweep to level 2 (Eq. (43)) -> M2L on every
      level 2..D over the interaction lists (Eq. (45)) -> L2L downsweep
      (Eq. (48)) -> L2P at the leaves (Eq. (46)).
    lam and the result are in the caller's (original) order."""
    d, D = T["d"], T["D"]
    lam = np.asarray(lam, dtype=np.float64)
    ls = lam[T["perm"]]
    u_near = p2p(T, ls, kernel, eps)
    u_far = np.zeros(T["N"])
    if D >= 2:
        V = {D: p2m(T, ls, M, L)}
        for l in range(D, 2, -1):
            V[l - 1] = m2m(T, V[l], l, M, L)
        Lx = {l: np.zeros_like(V[l]) for l in range(2, D + 1)}
        for l in range(2, D + 1):
            m2l(T, V[l], Lx[l], l, omegaC, M, L)
        for l in range(3, D + 1):
            l2l(T, Lx[l - 1], Lx[l], l, M, L)
        l2p(T, Lx[D], M, L, u_far)
    us = u_near + u_far
    u = np.empty_like(us)
    u[T["perm"]] = us
    if return_parts:
        un = np.empty_like(us)
        un[T["perm"]] = u_near
        return u, un
    return u


def fmm_evaluate(X, lam, Y, lo, side: float, D: int, kernel: int, eps: float, omegaC, M: int,
                 L: float):
    """The FMM evaluation at new points Y (Eq. (1) with targets that are not centres):
    one tree over the centres followed by the new points (root cube [lo, lo+side]^d,
    depth D), coefficients lambda on the centres and 0 on the new points; the product
    at the new points.  Returns s[len(Y)]."""
    X = np.asarray(X, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    Z = np.concatenate([X, Y])
    lz = np.concatenate([np.asarray(lam, dtype=np.float64), np.zeros(len(Y))])
    T = tree(Z, lo, side, D)
    return fmm(T, lz, kernel, eps, omegaC, M, L)[len(X):]


def fmm_brute(T, lam, kernel: int, eps: float, omegaC, M: int, L: float):
    """Tiny-N brute force of what the FMM computes: Phi on near pairs, K on all others."""
    d = T["d"]
    xi, _ = freq_grid(M, L)
    nleaf = len(T["leaf_key"])
    near = np.zeros((nleaf, nleaf), dtype=np.uint8)
    for a in range(nleaf):
        near[a, T["near_idx"][T["near_off"][a]:T["near_off"][a + 1]]] = 1
    leaf_of = np.repeat(np.arange(nleaf, dtype=np.int64), np.diff(T["leaf_off"]))
    ls = np.ascontiguousarray(np.asarray(lam, dtype=np.float64)[T["perm"]])
    us = np.zeros(T["N"])
    lib().orc_fmm_brute(_I(d), _I(M), _p(xi), _p(np.ascontiguousarray(omegaC)), _L(T["N"]),
                        _p(T["xs"]), _p(ls), _p(leaf_of), _L(nleaf), _p(near), _I(kernel),
                        _D(eps), _p(us))
    u = np.empty_like(us)
    u[T["perm"]] = us
    return u


def global_G(T, lam, M: int, L: float):
    d = T["d"]
    xi, _ = freq_grid(M, L)
    ls = np.ascontiguousarray(np.asarray(lam, dtype=np.float64)[T["perm"]])
    G = np.zeros(n_modes(d, M), dtype=np.complex128)
    lib().orc_global_G(_I(d), _I(M), _p(xi), _L(T["N"]), _p(T["xs"]), _p(ls), _p(G))
    return G


def fmm_at_targets(T, lam, kernel: int, eps: float, omegaC, M: int, L: float, targets, G=None):
    """FMM output at selected targets (original indices), from u = near Phi + far K."""
    d = T["d"]
    xi, _ = freq_grid(M, L)
    if G is None:
        G = global_G(T, lam, M, L)
    ls = np.ascontiguousarray(np.asarray(lam, dtype=np.float64)[T["perm"]])
    inv = np.empty(T["N"], dtype=np.int64)
    inv[T["perm"]] = np.arange(T["N"])
    t_point = np.ascontiguousarray(inv[np.asarray(targets, dtype=np.int64)])
    t_leaf = np.ascontiguousarray(np.searchsorted(T["leaf_off"], t_point, side="right") - 1)
    u = np.zeros(len(t_point))
    lib().orc_fmm_at_targets(_I(d), _I(M), _p(xi), _p(np.ascontiguousarray(omegaC)), _p(G),
                             _p(T["leaf_off"]), _p(T["near_off"]), _p(T["near_idx"]), _p(T["xs"]),
                             _p(ls), _I(kernel), _D(eps), _L(len(t_point)), _p(t_point),
                             _p(t_leaf.astype(np.int64)), _p(u))
    return u
