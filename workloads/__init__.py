"""Seeded synthetic inputs shaped like the paper's RBF workloads.

This module only draws random numbers; it holds none of the method's
arithmetic.  Both the CUDA-path tests/bench and the CPU oracle take their
inputs from here.  Draw order for every configuration: centres, then
coefficients or data values, then sampled target indices.  Exact duplicate
centres are removed (first occurrence kept) so that the interpolation matrix
stays non-singular.

The paper uses no public dataset; these generators stand in for "quasi-uniform
centres X in a bounded domain" (Sec. 1, Eq. (1)) at the sizes of the
benchmark configurations.
"""
from __future__ import annotations

import numpy as np


def _dedup(X):
    _, first = np.unique(X, axis=0, return_index=True)
    if len(first) == len(X):
        return X
    return X[np.sort(first)]


def config1():
    """d=2, N=4096 uniform in [0,1]^2 (seed 0), Gaussian eps=4, lambda ~ N(0,1), depth 3."""
    rng = np.random.default_rng(0)
    X = _dedup(rng.random((4096, 2)))
    lam = rng.standard_normal(len(X))
    params = dict(kernel=0, eps=4.0, depth=3, M=32, L=2.5, alpha=0.0, d=2)
    return X, lam, params


def config2(n=1 << 20, n_targets=4096):
    """d=3, N=2^20 uniform in [0,1]^3 (seed 1), inverse multiquadric eps=2,
    lambda ~ N(0,1), depth 5 (32 points per leaf on average), 4096 sampled targets."""
    rng = np.random.default_rng(1)
    X = _dedup(rng.random((n, 3)))
    lam = rng.standard_normal(len(X))
    targets = rng.choice(len(X), size=min(n_targets, len(X)), replace=False)
    depth = max(2, int(round(np.log(len(X) / 32.0) / np.log(8.0))))
    params = dict(kernel=1, eps=2.0, depth=depth, M=32, L=4.0, alpha=4.5, d=3)
    return X, lam, targets, params


def config3(n=262144):
    """d=3 clustered centres: mixture of 8 isotropic Gaussians (sd 0.05, means uniform in
    [0.2,0.8]^3), clipped to the cube (seed 2); Gaussian eps=3; data
    u = sin(2 pi x) cos(2 pi y) exp(-z)."""
    rng = np.random.default_rng(2)
    means = rng.uniform(0.2, 0.8, (8, 3))
    comp = rng.integers(8, size=n)
    X = np.clip(means[comp] + 0.05 * rng.standard_normal((n, 3)), 0.0, 1.0)
    X = _dedup(X)
    u = np.sin(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1]) * np.exp(-X[:, 2])
    params = dict(kernel=0, eps=3.0, M=24, L=3.0, alpha=0.0, d=3)
    return X, u, params


def config4(n_problems=256):
    """256 independent problems: N log-uniform in [2048, 65536], d in {2,3}, uniform
    centres, Gaussian or IMQ with eps ~ U[1,5], 4 right-hand sides ~ N(0,1) (seed 3)."""
    rng = np.random.default_rng(3)
    probs = []
    for _ in range(n_problems):
        N = int(round(np.exp(rng.uniform(np.log(2048), np.log(65536)))))
        d = int(rng.choice([2, 3]))
        kernel = int(rng.integers(2))
        eps = float(rng.uniform(1.0, 5.0))
        X = _dedup(rng.random((N, d)))
        U = rng.standard_normal((len(X), 4))
        probs.append(dict(X=X, U=U, d=d, kernel=kernel, eps=eps))
    return probs


def config5(n=1 << 19, n_targets=2048, nrhs=16):
    """d=5, N=2^19 uniform in [0,1]^5 (seed 4), Gaussian eps=1.5, lambda ~ N(0,1) plus a
    16-column lambda block, 2048 sampled targets."""
    rng = np.random.default_rng(4)
    X = _dedup(rng.random((n, 5)))
    lam = rng.standard_normal(len(X))
    lam_block = rng.standard_normal((len(X), nrhs))
    targets = rng.choice(len(X), size=min(n_targets, len(X)), replace=False)
    params = dict(kernel=0, eps=1.5, depth=2, M=12, L=4.0, alpha=0.0, d=5)
    return X, lam, lam_block, targets, params


def uniform(n, d, seed):
    """Generic small case: n uniform centres in [0,1]^d and lambda ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    X = _dedup(rng.random((n, d)))
    lam = rng.standard_normal(len(X))
    return X, lam


def jittered_grid(n1, d, seed, jitter=0.3):
    """Quasi-uniform centres: the n1^d cell centres of a regular grid on [0,1]^d, each
    moved by a uniform offset of at most jitter/2 cells per coordinate (seeded)."""
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(*[np.arange(n1)] * d, indexing="ij"), -1).reshape(-1, d)
    return (g + 0.5 + jitter * rng.uniform(-0.5, 0.5, g.shape)) / n1
