"""GPU parity of the MLFMM on nested (scale-invariant) frequency grids.

rbf_fmm_matvec with grid = RBF_GRID_NESTED runs M2M by Lagrange interpolation
in xi, M2L per level with that level's coefficients and L2L by anterpolation
(Sec. 4.1, 4.1.1).  Every case is compared element by element with the FP64
oracle of ``oracle/nested.py`` on the same tree: FP64 to 1e-12 (relative L2 and
every element relative to max |u_ref|), FP32 to 5e-6 relative L2 and 1.5e-5
element-wise.  The FP32 element bound is wider than on the shared grid
because every level adds 2 d interpolation passes (Lagrange stencils of K
taps, Eqs. (43), (48)) whose weights exceed 1 in magnitude and amplify the
rounding of the passes before them (measured: 6.5e-6 on the clustered 2-D
case against 3e-7 on the shared grid).  The cases span d = 1, 2, 3, several mode chunks per box, both
kernels, stencils of 4, 8 and 12 points, clustered points (empty boxes,
ragged leaves), depth 2 (no interpolation at all) and M = 40 (lines of 41
nodes along each dimension).
"""
import numpy as np
import pytest

import oracle as O
import workloads
from _parity import errs, rel
from oracle import nested as ON

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 5e-6        # relative L2
FP32_MAX_TOL = 1.5e-5  # element-wise, relative to max |u_ref|


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


def _clustered(n, d, seed):
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.2, 0.8, (3, d))
    return np.clip(means[rng.integers(3, size=n)] + 0.05 * rng.standard_normal((n, d)), 0, 1)


CASES = [
    # name, d, N, D, kernel, eps, M, K, kind
    ("1d-depth5-K8", 1, 3000, 5, O.IMQ, 2.0, 16, 8, "u"),
    ("2d-depth4-K8", 2, 5000, 4, O.IMQ, 2.0, 16, 8, "u"),
    ("2d-gauss-K4", 2, 4000, 3, O.GAUSSIAN, 3.0, 12, 4, "u"),
    ("2d-clustered-K8", 2, 4000, 4, O.IMQ, 2.0, 16, 8, "c"),
    ("3d-depth3-K8", 3, 6000, 3, O.IMQ, 2.0, 16, 8, "u"),
    ("3d-M24-K12", 3, 3000, 3, O.GAUSSIAN, 2.0, 24, 12, "u"),
    ("3d-depth2", 3, 2000, 2, O.IMQ, 2.0, 16, 8, "u"),
    # 3-D M = 40 (41 nodes per dimension: more than one warp per line)
    ("3d-M40", 3, 600, 3, O.IMQ, 2.0, 40, 8, "u"),
]


@pytest.mark.parametrize("name,d,n,D,kernel,eps,M,K,kind", CASES)
def test_nested_matches_oracle(rbf, name, d, n, D, kernel, eps, M, K, kind):
    import torch
    X = _clustered(n, d, n + d) if kind == "c" else workloads.uniform(n, d, seed=n + 3 * d)[0]
    lam = np.random.default_rng(n + D).standard_normal(len(X))
    T = O.tree(X, np.zeros(d), 1.0, D)
    wcs = ON.coeffs_levels(kernel, eps, d, M, 4.0, 4.5, 1.0, D)
    ref = ON.fmm(T, lam, kernel, eps, wcs, M, 4.0, K)
    t = rbf.tree_build(_dev(X), lo=np.zeros(d), side=1.0, depth=D)
    out = {}
    for prec in (rbf.FP64, rbf.FP32):
        u = torch.empty(len(X), dtype=torch.float64, device="cuda")
        rbf.fmm_matvec(t, kernel, eps, _dev(lam), u, prec=prec, M=M, period_L=4.0, window_alpha=4.5,
                       grid=rbf.GRID_NESTED, lagrange_K=K)
        torch.cuda.synchronize()
        out[prec] = u.cpu().numpy()
    e64, e32 = rel(out[rbf.FP64], ref), errs(out[rbf.FP32], ref)
    print(f"{name}: FP64 {e64:.2e}, FP32 rel-L2 {e32[0]:.2e} max {e32[1]:.2e} vs the nested oracle")
    assert e64 <= FP64_TOL
    assert e32[0] <= FP32_TOL and e32[1] <= FP32_MAX_TOL


def test_nested_depth2_equals_shared_grid_on_device(rbf):
    """At depth 2 the nested product is the shared-grid product (same level-2
    grid and coefficients): the two device paths agree to rounding."""
    import torch
    X, _ = workloads.uniform(3000, 2, 77)
    lam = _dev(np.random.default_rng(78).standard_normal(3000))
    t = rbf.tree_build(_dev(X), lo=np.zeros(2), side=1.0, depth=2)
    kw = dict(prec=rbf.FP64, M=16, period_L=4.0, window_alpha=4.5)
    a = torch.empty(3000, dtype=torch.float64, device="cuda")
    b = torch.empty_like(a)
    rbf.fmm_matvec(t, O.IMQ, 2.0, lam, a, **kw)
    rbf.fmm_matvec(t, O.IMQ, 2.0, lam, b, grid=rbf.GRID_NESTED, lagrange_K=8, **kw)
    torch.cuda.synchronize()
    assert rel(b.cpu().numpy(), a.cpu().numpy()) < 1e-13


def test_nested_several_columns_and_plan_switch(rbf):
    """Several right-hand sides on nested grids run column by column and equal
    single-column products; switching a tree between the shared and nested
    plans gives the same results as fresh plans."""
    import torch
    X, _ = workloads.uniform(4000, 3, 91)
    lam = np.random.default_rng(92).standard_normal((5, 4000))
    t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=3)
    kw = dict(prec=rbf.FP32, M=16, period_L=4.0, window_alpha=4.5)
    U = torch.empty(5, 4000, dtype=torch.float64, device="cuda")
    rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), U, grid=rbf.GRID_NESTED, **kw)
    S = torch.empty_like(U)
    rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), S, **kw)
    U1 = torch.empty_like(U)
    for c in range(5):
        rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam[c]), U1[c], grid=rbf.GRID_NESTED, **kw)
    torch.cuda.synchronize()
    assert torch.equal(U, U1)
    # both grids approximate the same product
    assert rel(U.cpu().numpy(), S.cpu().numpy()) < 1e-3


def test_nested_rejects_unsupported(rbf):
    """d > 3 is not built (RBF_ENOTSUP); no taper, closed-form coefficients,
    an odd stencil or M < 2K are argument errors."""
    import torch
    X4, _ = workloads.uniform(500, 4, 5)
    t4 = rbf.tree_build(_dev(X4), lo=np.zeros(4), side=1.0, depth=2)
    u = torch.empty(500, dtype=torch.float64, device="cuda")
    lam = _dev(np.ones(500))
    with pytest.raises(rbf.RbfError) as e:
        rbf.fmm_matvec(t4, O.IMQ, 2.0, lam, u, M=16, grid=rbf.GRID_NESTED)
    assert e.value.code == -6
    X, _ = workloads.uniform(500, 2, 6)
    t = rbf.tree_build(_dev(X), lo=np.zeros(2), side=1.0, depth=3)
    bad = [dict(M=16, window_alpha=0.0), dict(M=16, csample=0, window_alpha=4.5),
           dict(M=16, lagrange_K=5, window_alpha=4.5), dict(M=12, lagrange_K=8, window_alpha=4.5)]
    for kw in bad:
        with pytest.raises(rbf.RbfError) as e:
            rbf.fmm_matvec(t, O.GAUSSIAN, 2.0, lam, u, grid=rbf.GRID_NESTED, **kw)
        assert e.value.code == -1


def test_nested_full_size_3d(rbf):
    """3-D, N = 2^20, depth 5 (32 points per leaf), M = 32, K = 8: the FP32
    product matches the FP64 product to the FP32 bound, and both approximate the
    direct sum at sampled targets as closely as the shared-grid product does
    (within a factor 2 of its error)."""
    import torch
    n = 1 << 20
    X, lam = workloads.uniform(n, 3, 2024)
    t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=5)
    kw = dict(M=32, period_L=4.0, window_alpha=4.5)
    lam_d = _dev(lam)
    res = {}
    for name, prec, grid in (("n64", rbf.FP64, rbf.GRID_NESTED), ("n32", rbf.FP32, rbf.GRID_NESTED),
                             ("s32", rbf.FP32, rbf.GRID_SHARED)):
        u = torch.empty(n, dtype=torch.float64, device="cuda")
        rbf.fmm_matvec(t, O.IMQ, 2.0, lam_d, u, prec=prec, grid=grid, **kw)
        torch.cuda.synchronize()
        res[name] = u
    assert rel(res["n32"].cpu().numpy(), res["n64"].cpu().numpy()) < FP32_TOL
    tg = np.random.default_rng(9).choice(n, 1024, replace=False)
    ud = O.direct(X, lam, O.IMQ, 2.0, targets=tg)
    e_nested = rel(res["n64"].cpu().numpy()[tg], ud)
    e_shared = rel(res["s32"].cpu().numpy()[tg], ud)
    print(f"3d N=2^20 vs direct (1024 targets): nested FP64 {e_nested:.2e}, shared FP32 {e_shared:.2e}")
    assert e_nested <= 2.0 * e_shared + 1e-7
