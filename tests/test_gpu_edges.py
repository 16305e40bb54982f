"""Degenerate and extreme inputs of the product on the GPU.

Each case is compared element by element with the FP64 oracle FMM on the same
tree (FP64 to 1e-12 relative L2, FP32 to 5e-6) and, where the answer has a
closed form, with that too:

* one centre (u = Phi(0) lambda), at depth 0 and at depth 3;
* 2000 coincident centres: one leaf holds every point, the far field of a
  lone leaf cancels, and u_i = Phi(0) sum_j lambda_j for every i (Eq. (1));
* one crowded leaf of 3000 points among 1000 uniform ones (many phase-table
  chunks in one CTA, a near list dominated by one leaf);
* the largest expansion (M = 64, 65 columns) and the smallest (M = 2);
* leaves of at most a few points at depth 7;
* zero coefficients give exactly zero; N = 0 is an argument error.

The coefficients are positive (uniform in [0.5, 1.5]): with thousands of nearly
coincident centres and random signs, u_i would be a cancelling sum whose FP32
rounding is set by sum|lambda| / |sum lambda|, not by the method.
"""
import numpy as np
import pytest

import oracle as O
import workloads
from _parity import rel

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 5e-6


@pytest.fixture(scope="module")
def rbf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_07652_gb300 as m
    m.load()
    return m


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def _crowded(seed):
    rng = np.random.default_rng(seed)
    A = 0.53 + 0.004 * rng.random((3000, 3))
    B, _ = workloads.uniform(1000, 3, seed + 1)
    return np.concatenate([A, B])


CASES = [
    # name, X, D, kernel, eps, M, L, alpha
    ("single-2d-depth0", np.array([[0.3, 0.7]]), 0, O.IMQ, 2.0, 8, 4.0, 4.5),
    ("single-3d-depth3", np.array([[0.3, 0.7, 0.1]]), 3, O.GAUSSIAN, 3.0, 8, 3.0, 0.0),
    ("coincident-3d", np.tile([[0.41, 0.77, 0.13]], (2000, 1)), 4, O.IMQ, 2.0, 12, 4.0, 4.5),
    ("crowded-leaf-3d", _crowded(3), 4, O.IMQ, 2.0, 12, 4.0, 4.5),
    ("max-M-3d", workloads.uniform(1500, 3, 7)[0], 2, O.IMQ, 2.0, 64, 4.0, 4.5),
    ("min-M-2d", workloads.uniform(2000, 2, 8)[0], 3, O.GAUSSIAN, 3.0, 2, 3.0, 0.0),
    ("deep-2d-depth7", workloads.uniform(400, 2, 9)[0], 7, O.IMQ, 2.0, 8, 4.0, 4.5),
]


@pytest.mark.parametrize("name,X,D,kernel,eps,M,L,alpha", CASES, ids=[c[0] for c in CASES])
def test_edge_matches_oracle(rbf, name, X, D, kernel, eps, M, L, alpha):
    import torch
    d = X.shape[1]
    lam = np.random.default_rng(len(X)).uniform(0.5, 1.5, len(X))
    T = O.tree(X, np.zeros(d), 1.0, D)
    wc = O.coeffs_sampled(kernel, eps, d, M, L, alpha, 1.0)
    ref = O.fmm(T, lam, kernel, eps, wc, M, L)
    t = rbf.tree_build(_dev(X), lo=np.zeros(d), side=1.0, depth=D)
    lam_d = _dev(lam)
    out = {}
    for prec in (rbf.FP64, rbf.FP32):
        u = torch.empty_like(lam_d)
        rbf.fmm_matvec(t, kernel, eps, lam_d, u, prec=prec, M=M, period_L=L, window_alpha=alpha)
        torch.cuda.synchronize()
        out[prec] = u.cpu().numpy()
    e64, e32 = rel(out[rbf.FP64], ref), rel(out[rbf.FP32], ref)
    print(f"{name}: FP64 {e64:.2e}, FP32 {e32:.2e} vs the oracle")
    assert e64 <= FP64_TOL
    assert e32 <= FP32_TOL
    phi0 = float(O.phi(kernel, eps, np.zeros(1))[0])
    if len(X) == 1 or name.startswith("coincident"):
        # every pair is at distance 0: u_i = Phi(0) sum_j lambda_j
        exact = np.full(len(X), phi0 * lam.sum())
        assert rel(out[rbf.FP64], exact) <= FP64_TOL
        assert rel(out[rbf.FP32], exact) <= FP32_TOL
    if name.startswith("max-M"):
        # 65 nodes per dimension resolve the IMQ kernel: the product is the direct sum
        assert rel(out[rbf.FP64], O.direct(X, lam, kernel, eps)) <= 1e-10


def test_zero_coefficients_give_zero(rbf):
    import torch
    X, _ = workloads.uniform(3000, 3, 12)
    t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=3)
    lam = torch.zeros(3000, dtype=torch.float64, device="cuda")
    for prec in (rbf.FP64, rbf.FP32):
        u = torch.full_like(lam, np.nan)
        rbf.fmm_matvec(t, O.IMQ, 2.0, lam, u, prec=prec, M=12, period_L=4.0, window_alpha=4.5)
        torch.cuda.synchronize()
        assert torch.count_nonzero(u).item() == 0


def test_empty_input_is_an_argument_error(rbf):
    import torch
    X = torch.empty((0, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(rbf.RbfError) as e:
        rbf.tree_build(X, lo=np.zeros(3), side=1.0, depth=2)
    assert e.value.code == -1
