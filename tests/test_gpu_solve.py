"""GPU interpolation solve (GMRES + FP64 refinement) against the oracle.

Problem: 576 centres on a jittered 24 x 24 grid in [0,1]^2, Gaussian eps=20
(condition number ~3e2), data u = sin(2 pi x) cos(2 pi y), quadtree depth 3,
M=64, L=1.3 (far-kernel error ~4e-8).  Residuals are checked with the oracle's
own FP64 FMM product, so they measure the solve, not the GPU product."""
import numpy as np
import pytest

import oracle as O
from oracle.solver import gmres

pytestmark = pytest.mark.gpu

EPS, M, L, D = 20.0, 64, 1.3, 3


def _problem():
    rng = np.random.default_rng(3)
    n1 = 24
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij"), -1).reshape(-1, 2)
    X = (g + 0.5 + 0.3 * rng.uniform(-0.5, 0.5, (n1 * n1, 2))) / n1
    u = np.sin(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1])
    return X, u


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_07652_gb300 as rbf
    X, u = _problem()
    T = O.tree(X, np.zeros(2), 1.0, D)
    wc = O.coeffs_sampled(O.GAUSSIAN, EPS, 2, M, L, 0.0, 1.0)
    A = lambda v: O.fmm(T, v, O.GAUSSIAN, EPS, wc, M, L)
    t = rbf.tree_build(torch.as_tensor(X, device="cuda"), lo=np.zeros(2), side=1.0, depth=D)
    return rbf, torch, X, u, A, t


def _solve(setup, **kw):
    rbf, torch, X, u, A, t = setup
    ud = torch.as_tensor(u, device="cuda")
    lam = torch.zeros_like(ud)
    rep = rbf.interp_solve(t, rbf.GAUSSIAN, EPS, ud, lam, M=M, period_L=L, window_alpha=0.0, **kw)
    return rep, lam.cpu().numpy()


@pytest.mark.parametrize("inner", ["fp64", "fp32"])
def test_solve_reaches_tolerance(setup, inner):
    rbf, torch, X, u, A, t = setup
    prec = rbf.FP64 if inner == "fp64" else rbf.FP32
    rep, lam = _solve(setup, rtol=1e-9, restart_m=50, max_iters=3000, max_refine=8,
                      inner_prec=prec)
    assert rep["status"] == 0, rep
    assert rep["rel_resid"] <= 1e-9
    res = np.linalg.norm(u - A(lam)) / np.linalg.norm(u)
    assert res <= 1.5e-9, res
    if inner == "fp32":
        assert rep["refinements"] >= 2 and rep["matvecs_fp64"] >= 2


def test_fp64_iteration_count_matches_oracle_gmres(setup):
    """Same operator (parity 1e-15), same restart length and stopping rule: the GPU
    GMRES takes the oracle's number of iterations (one refinement step)."""
    rbf, torch, X, u, A, t = setup
    rep, lam = _solve(setup, rtol=1e-9, restart_m=50, max_iters=3000, max_refine=3,
                      inner_prec=rbf.FP64)
    _, it, _ = gmres(A, u, m=50, tol=0.5e-9, maxit=3000)
    assert abs(rep["iters"] - it) <= 2, (rep["iters"], it)


def test_nonconvergence_is_reported(setup):
    rbf, torch, X, u, A, t = setup
    rep, lam = _solve(setup, rtol=1e-12, restart_m=10, max_iters=5, max_refine=2,
                      inner_prec=rbf.FP64)
    assert rep["status"] == -4
    assert rep["rel_resid"] > 1e-12
    assert np.all(np.isfinite(lam))
