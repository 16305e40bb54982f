"""Error measures shared by the GPU parity tests.

Every comparison against the oracle bounds two numbers with the same
tolerance: the relative L2 error over the whole output, and the element-wise
error max_i |got_i - ref_i| / max_i |ref_i|.  The second catches one wrong
leaf (or one wrong point) that a relative L2 over many points would dilute.
"""
import numpy as np


def errs(got, ref):
    """(relative L2 error, max-norm error relative to max |ref|) of got against ref."""
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert got.shape == ref.shape, (got.shape, ref.shape)
    diff = got - ref
    nref, mref = np.linalg.norm(ref), np.max(np.abs(ref)) if ref.size else 0.0
    if nref == 0.0:
        z = 0.0 if not np.any(diff) else float("inf")
        return z, z
    return float(np.linalg.norm(diff) / nref), float(np.max(np.abs(diff)) / mref)


def rel(got, ref):
    """The worse of the two measures in errs(): a test asserting rel(...) <= tol
    bounds both the relative L2 error and every element's error by tol * max|ref|."""
    l2, mx = errs(got, ref)
    return max(l2, mx)


def spread_sample(leaf_off, rng, n_random=160, keys=None, d=None, depth=None):
    """Sorted-order point indices that reach leaves of every occupancy.

    For each distinct leaf size, the first and the last point of one leaf of
    that size (the last point lies in a later point chunk of a kernel that
    splits large leaves); every point of the most crowded leaf; when the leaf
    keys are given, the first point of up to 32 leaves on the root cube's
    boundary; then n_random uniform picks."""
    leaf_off = np.asarray(leaf_off, dtype=np.int64)
    occ = np.diff(leaf_off)
    picks = []
    for size in np.unique(occ[occ > 0]):
        leaves = np.flatnonzero(occ == size)
        a = int(rng.choice(leaves))
        picks += [leaf_off[a], leaf_off[a + 1] - 1]
    big = int(np.argmax(occ))
    picks += list(range(leaf_off[big], leaf_off[big + 1]))
    if keys is not None:
        keys = np.asarray(keys, dtype=np.uint64)
        coords = np.zeros((len(keys), d), dtype=np.int64)
        for b in range(depth):
            for t in range(d):
                coords[:, t] |= ((keys >> np.uint64(b * d + t)) & np.uint64(1)).astype(np.int64) << b
        edge = np.flatnonzero(np.any((coords == 0) | (coords == (1 << depth) - 1), axis=1)
                              & (occ > 0))
        for a in rng.choice(edge, size=min(32, len(edge)), replace=False):
            picks.append(leaf_off[a])
    picks += list(rng.choice(leaf_off[-1], size=n_random, replace=False))
    return np.unique(np.asarray(picks, dtype=np.int64))
