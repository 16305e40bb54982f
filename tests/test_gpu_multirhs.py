"""GPU parity of the multi-right-hand-side FP32 product (tensor-core P2M/L2P).

With RBF_FP32 and at least four columns, rbf_fmm_matvec runs P2M and L2P of
several columns as complex matrix products on the tensor cores (three-term
split TF32 operands, FP32 accumulation).  Every column must match the FP64
oracle FMM, and the single-column FP32 product, to the FP32 bound of the
single-column tests in relative L2 (5e-6).  Element by element the bound is
1.5e-5 of max |u_ref|: the split x = hi + lo with hi, lo in TF32 keeps about
22 significant bits (2^-21 per product against 2^-24 for FP32 arithmetic), and
the tensor core's accumulation rounds towards zero over each 12-MMA block, so
the worst element of this path carries about 20x the error of the CUDA-core
path (measured 6e-6 against 3e-7).  The cases cover several row and column
tiles, several point tiles per leaf (leaves above 128 points), d = 1, 2, 3, 5,
ragged clustered leaves, and more columns than one group holds.
"""
import numpy as np
import pytest

import oracle as O
import workloads
from _parity import errs

pytestmark = pytest.mark.gpu

FP32_TOL = 5e-6        # relative L2
TC_MAX_TOL = 1.5e-5    # element-wise, relative to max |u_ref| (tensor-core operand split)


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
    means = rng.uniform(0.2, 0.8, (4, d))
    return np.clip(means[rng.integers(4, size=n)] + 0.03 * rng.standard_normal((n, d)), 0, 1)


# Leaves of at least 64 points send P2M to the tensor cores, at least 96 also
# L2P; smaller leaves take the CUDA-core kernels column by column.  The near
# field of a group always runs as one multi-column pass.
CASES = [
    # name, d, N, D, kernel, eps, M, L, alpha, R, kind
    ("3d-row-col-point-tiles", 3, 12000, 2, O.IMQ, 2.0, 16, 4.0, 4.5, 16, "u"),
    ("config1-shape-R4", 2, 4096, 3, O.GAUSSIAN, 4.0, 32, 2.5, 0.0, 4, "u"),
    ("1d-R6", 1, 3000, 4, O.IMQ, 3.0, 24, 4.0, 4.5, 6, "u"),
    ("2d-two-groups-R20", 2, 6000, 2, O.IMQ, 2.0, 16, 4.0, 4.5, 20, "u"),
    ("3d-clustered-ragged-R5", 3, 6000, 2, O.GAUSSIAN, 3.0, 10, 3.0, 0.0, 5, "c"),
    ("2d-small-leaves-R8", 2, 3000, 3, O.IMQ, 2.0, 16, 4.0, 4.5, 8, "u"),
    ("2d-mq-R6", 2, 6000, 2, O.MQ, 2.0, 16, 4.0, 4.5, 6, "u"),
    ("3d-wendland-R4", 3, 12000, 2, O.WENDLAND, 0.5, 12, 4.0, 0.0, 4, "u"),
]


@pytest.mark.parametrize("name,d,n,D,kernel,eps,M,L,alpha,R,kind", CASES)
def test_multi_rhs_matches_oracle_and_single_column(rbf, name, d, n, D, kernel, eps, M, L, alpha,
                                                    R, kind):
    import torch
    if name.startswith("config1"):
        X, _, _ = workloads.config1()
    elif kind == "c":
        X = _clustered(n, d, seed=n)
    else:
        X, _ = workloads.uniform(n, d, seed=n + d)
    lam = np.random.default_rng(100 + R).standard_normal((R, len(X)))
    T = O.tree(X, np.zeros(d), 1.0, D)
    wc = O.coeffs_sampled(kernel, eps, d, M, L, alpha, 1.0)
    t = rbf.tree_build(_dev(X), lo=np.zeros(d), side=1.0, depth=D)
    kw = dict(prec=rbf.FP32, M=M, period_L=L, window_alpha=alpha)
    lam_d = _dev(lam)
    U = torch.empty_like(lam_d)
    rbf.fmm_matvec(t, kernel, eps, lam_d, U, **kw)
    Us = torch.empty_like(lam_d)
    for c in range(R):
        rbf.fmm_matvec(t, kernel, eps, lam_d[c], Us[c], **kw)
    torch.cuda.synchronize()
    rbf.check_device_waits()
    U = U.cpu().numpy()
    Us = Us.cpu().numpy()
    worst_o, worst_s = np.zeros(2), np.zeros(2)
    occ = np.diff(T["leaf_off"])
    where = None
    for c in range(R):
        ref = O.fmm(T, lam[c], kernel, eps, wc, M, L)
        eo = np.array(errs(U[c], ref))
        if eo[1] > worst_o[1]:
            i = int(np.argmax(np.abs(U[c] - ref)))
            pos = int(np.flatnonzero(T["perm"] == i)[0])
            leaf = int(np.searchsorted(T["leaf_off"], pos, side="right") - 1)
            where = (c, leaf, int(occ[leaf]))
        worst_o = np.maximum(worst_o, eo)
        worst_s = np.maximum(worst_s, errs(U[c], Us[c]))
    print(f"{name}: R={R} vs oracle rel-L2 {worst_o[0]:.2e} max {worst_o[1]:.2e} "
          f"(column, leaf, leaf size {where}); vs single-column FP32 rel-L2 {worst_s[0]:.2e} "
          f"max {worst_s[1]:.2e}")
    assert worst_o[0] <= FP32_TOL and worst_o[1] <= TC_MAX_TOL
    assert worst_s[0] <= FP32_TOL and worst_s[1] <= TC_MAX_TOL


def test_multi_rhs_repeatable_and_leading_columns_independent(rbf):
    """The same call twice gives the same bits; a column's result does not
    depend on the other columns of its group."""
    import torch
    X, _ = workloads.uniform(6000, 3, 31)
    lam = np.random.default_rng(5).standard_normal((8, len(X)))
    t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=3)
    kw = dict(prec=rbf.FP32, M=12, period_L=4.0, window_alpha=4.5)
    lam_d = _dev(lam)
    U1 = torch.empty_like(lam_d)
    U2 = torch.empty_like(lam_d)
    rbf.fmm_matvec(t, O.IMQ, 2.0, lam_d, U1, **kw)
    rbf.fmm_matvec(t, O.IMQ, 2.0, lam_d, U2, **kw)
    lam_b = lam.copy()
    lam_b[1:] = np.random.default_rng(6).standard_normal((7, len(X)))
    U3 = torch.empty_like(lam_d)
    rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam_b), U3, **kw)
    torch.cuda.synchronize()
    rbf.check_device_waits()
    assert torch.equal(U1, U2)
    assert torch.equal(U1[0], U3[0])


def test_multi_rhs_5d_tensor_core_sampled(rbf):
    """d = 5, N = 2^17 (128 points per leaf at depth 2, so both contractions
    run on the tensor cores), 16 columns: every column against the
    single-column FP32 product, four columns against the oracle's FMM output
    at sampled targets (oracle.fmm_at_targets)."""
    import torch
    X, _ = workloads.uniform(1 << 17, 5, 55)
    R, M, L, eps = 16, 4, 4.0, 1.5
    lam = np.random.default_rng(56).standard_normal((R, len(X)))
    t = rbf.tree_build(_dev(X), lo=np.zeros(5), side=1.0, depth=2)
    kw = dict(prec=rbf.FP32, M=M, period_L=L, window_alpha=0.0)
    lam_d = _dev(lam)
    U = torch.empty_like(lam_d)
    rbf.fmm_matvec(t, O.GAUSSIAN, eps, lam_d, U, **kw)
    Us = torch.empty_like(lam_d)
    for c in range(R):
        rbf.fmm_matvec(t, O.GAUSSIAN, eps, lam_d[c], Us[c], **kw)
    torch.cuda.synchronize()
    rbf.check_device_waits()
    U = U.cpu().numpy()
    Us = Us.cpu().numpy()
    worst_s = np.max([errs(U[c], Us[c]) for c in range(R)], axis=0)
    T = O.tree(X, np.zeros(5), 1.0, 2)
    wc = O.coeffs_sampled(O.GAUSSIAN, eps, 5, M, L, 0.0, 1.0)
    sample = np.random.default_rng(57).choice(len(X), size=64, replace=False)
    worst_o = np.zeros(2)
    for c in (0, 5, 10, 15):
        ref = O.fmm_at_targets(T, lam[c], O.GAUSSIAN, eps, wc, M, L, sample)
        worst_o = np.maximum(worst_o, errs(U[c][sample], ref))
    print(f"5d N=2^17 R=16: vs oracle (sampled) rel-L2 {worst_o[0]:.2e} max {worst_o[1]:.2e}; "
          f"vs single-column rel-L2 {worst_s[0]:.2e} max {worst_s[1]:.2e}")
    assert worst_o[0] <= FP32_TOL and worst_o[1] <= TC_MAX_TOL
    assert worst_s[0] <= FP32_TOL and worst_s[1] <= TC_MAX_TOL
