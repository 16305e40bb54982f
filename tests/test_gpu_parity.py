"""GPU parity: the sm_103a library against the FP64 CPU oracle, element by element.

Tree, permutation and lists must be bit-exact.  The FP64 product must match the
oracle's multilevel FMM to 1e-12; the FP32 product is held to a stated bound
(5e-6, about 80 FP32 ulps of accumulated rounding, well under the method's own
kernel error at these expansion sizes).  Each bound applies both to the
relative L2 error and to every element's error relative to max |u_ref|
(tests/_parity.py).
"""
import os

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


def _clustered(n, d, seed):
    rng = np.random.default_rng(seed)
    means = rng.uniform(0.2, 0.8, (4, d))
    X = np.clip(means[rng.integers(4, size=n)] + 0.03 * rng.standard_normal((n, d)), 0, 1)
    return X, rng.standard_normal(n)


TREE_CASES = [
    ("uniform-2d", 2, 5000, 4, "u"),
    ("uniform-3d-ragged", 3, 7777, 3, "u"),
    ("clustered-3d-empty-leaves", 3, 6000, 5, "c"),
    ("faces-2d", 2, 700, 3, "f"),
    ("depth0", 2, 50, 0, "u"),
    ("depth1-1d", 1, 300, 1, "u"),
    ("5d", 5, 3000, 2, "u"),
]


def _points(d, n, kind, seed):
    if kind == "c":
        return _clustered(n, d, seed)
    X, lam = workloads.uniform(n, d, seed)
    if kind == "f":
        X[:50] = np.round(X[:50] * 8) / 8  # exactly on box faces
        X[50] = 1.0
        X[51] = 0.0
    return X, lam


@pytest.mark.parametrize("name,d,n,D,kind", TREE_CASES)
def test_tree_bit_exact(rbf, name, d, n, D, kind):
    X, _ = _points(d, n, kind, seed=len(name))
    T = O.tree(X, np.zeros(d), 1.0, D)
    t = rbf.tree_build(_dev(X), lo=np.zeros(d), side=1.0, depth=D)
    e = t.export()
    assert np.array_equal(e["perm"], T["perm"])
    assert np.array_equal(e["keys"], T["keys"])
    assert np.array_equal(e["leaf_key"], T["leaf_key"])
    assert np.array_equal(e["leaf_off"], T["leaf_off"])
    assert np.array_equal(e["near_off"], T["near_off"])
    assert np.array_equal(e["near_idx"], T["near_idx"])
    info = t.info()
    for l in range(D + 1):
        assert info["n_box"][l] == len(T["levels"][l]["key"])
    for l in range(2, D + 1):
        lv = t.export_level(l)
        assert np.array_equal(lv["key"], T["levels"][l]["key"])
        assert np.array_equal(lv["il_off"], T["levels"][l]["il_off"])
        assert np.array_equal(lv["il_idx"], T["levels"][l]["il_idx"])


MATVEC_CASES = [
    # name, d, N, D, kernel, eps, M, L, alpha, kind
    ("config1", 2, 4096, 3, O.GAUSSIAN, 4.0, 32, 2.5, 0.0, "u"),
    ("imq-3d-ragged", 3, 9000, 3, O.IMQ, 2.0, 12, 4.0, 4.5, "u"),
    ("imq-2d-deep", 2, 6000, 5, O.IMQ, 2.0, 16, 4.0, 4.5, "u"),
    ("gauss-3d-clustered", 3, 5000, 4, O.GAUSSIAN, 3.0, 10, 3.0, 0.0, "c"),
    ("near-only-depth1", 2, 800, 1, O.IMQ, 2.0, 8, 4.0, 4.5, "u"),
    ("depth2", 3, 2000, 2, O.GAUSSIAN, 3.0, 12, 3.0, 0.0, "u"),
    ("1d", 1, 3000, 4, O.IMQ, 3.0, 24, 4.0, 4.5, "u"),
    ("5d", 5, 1500, 2, O.GAUSSIAN, 1.5, 4, 4.0, 0.0, "u"),
    ("4d-depth3-grid", 4, 3000, 3, O.GAUSSIAN, 2.0, 6, 4.0, 0.0, "u"),
    ("6d", 6, 700, 2, O.IMQ, 1.0, 4, 4.0, 4.5, "u"),
    ("mq-2d", 2, 5000, 4, O.MQ, 2.0, 16, 4.0, 4.5, "u"),
    ("mq-3d-clustered", 3, 5000, 3, O.MQ, 1.0, 12, 4.0, 4.5, "c"),
    ("wendland-2d", 2, 5000, 4, O.WENDLAND, 0.5, 16, 4.0, 0.0, "u"),
    ("wendland-3d-taper", 3, 6000, 3, O.WENDLAND, 3.0, 12, 4.0, 4.5, "u"),
    ("wendland-1d", 1, 2000, 4, O.WENDLAND, 0.5, 16, 4.0, 0.0, "u"),
    # one dimension has M/2 + 1 columns: even counts (M = 2 mod 4) and the widest row
    ("1d-4-cols", 1, 2500, 4, O.GAUSSIAN, 2.0, 6, 3.0, 0.0, "u"),
    ("1d-16-cols", 1, 3000, 5, O.IMQ, 3.0, 30, 4.0, 4.5, "u"),
    ("1d-32-cols", 1, 2000, 3, O.GAUSSIAN, 3.0, 62, 3.0, 0.0, "u"),
]


@pytest.mark.parametrize("name,d,n,D,kernel,eps,M,L,alpha,kind", MATVEC_CASES)
def test_matvec_matches_oracle(rbf, name, d, n, D, kernel, eps, M, L, alpha, kind):
    import torch
    if name == "config1":
        X, lam, _ = workloads.config1()
    else:
        X, lam = _points(d, n, kind, seed=n)
    T = O.tree(X, np.zeros(d), 1.0, D)
    wc = O.coeffs_sampled(kernel, eps, d, M, L, alpha, 1.0)
    u_ref = O.fmm(T, lam, kernel, eps, wc, M, L)
    t = rbf.tree_build(_dev(X), lo=np.zeros(d), side=1.0, depth=D)
    lam_d = _dev(lam)
    u64 = torch.empty_like(lam_d)
    rbf.fmm_matvec(t, kernel, eps, lam_d, u64, prec=rbf.FP64, M=M, period_L=L, window_alpha=alpha)
    u32 = torch.empty_like(lam_d)
    rbf.fmm_matvec(t, kernel, eps, lam_d, u32, prec=rbf.FP32, M=M, period_L=L, window_alpha=alpha)
    torch.cuda.synchronize()
    e64 = rel(u64.cpu().numpy(), u_ref)
    e32 = rel(u32.cpu().numpy(), u_ref)
    print(f"{name}: fp64 rel {e64:.3e}  fp32 rel {e32:.3e}")
    assert e64 <= FP64_TOL
    assert e32 <= FP32_TOL
    # a second call reuses the cached plan and must give the same bits
    u64b = torch.empty_like(lam_d)
    rbf.fmm_matvec(t, kernel, eps, lam_d, u64b, prec=rbf.FP64, M=M, period_L=L, window_alpha=alpha)
    assert torch.equal(u64, u64b)


def test_closed_form_coefficients_gaussian(rbf):
    import torch
    X, lam = workloads.uniform(3000, 2, 9)
    T = O.tree(X, np.zeros(2), 1.0, 3)
    wc = O.coeffs_closed_gaussian(4.0, 2, 20, 2.5)
    u_ref = O.fmm(T, lam, O.GAUSSIAN, 4.0, wc, 20, 2.5)
    t = rbf.tree_build(_dev(X), lo=np.zeros(2), side=1.0, depth=3)
    u = torch.empty(len(X), dtype=torch.float64, device="cuda")
    rbf.fmm_matvec(t, O.GAUSSIAN, 4.0, _dev(lam), u, prec=rbf.FP64, M=20, period_L=2.5,
                   window_alpha=0.0, csample=0)
    assert rel(u.cpu().numpy(), u_ref) <= FP64_TOL


def test_multiple_rhs_and_host_entry(rbf):
    import torch
    X, lam = workloads.uniform(4000, 3, 21)
    rng = np.random.default_rng(4)
    lam2 = np.stack([lam, rng.standard_normal(len(X)), rng.standard_normal(len(X))])
    T = O.tree(X, np.zeros(3), 1.0, 3)
    wc = O.coeffs_sampled(O.IMQ, 2.0, 3, 10, 4.0, 4.5, 1.0)
    t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=3)
    U = torch.empty(lam2.shape, dtype=torch.float64, device="cuda")
    rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam2), U, prec=rbf.FP64, M=10, period_L=4.0)
    Uh = rbf.fmm_matvec_host(t, O.IMQ, 2.0, lam2, prec=rbf.FP64, M=10, period_L=4.0)
    for c in range(3):
        ref = O.fmm(T, lam2[c], O.IMQ, 2.0, wc, 10, 4.0)
        assert rel(U[c].cpu().numpy(), ref) <= FP64_TOL
        assert rel(Uh[c], ref) <= FP64_TOL


@pytest.mark.parametrize("kernel,eps", [(O.IMQ, 2.0), (O.GAUSSIAN, 3.0), (O.MQ, 2.0),
                                        (O.WENDLAND, 2.5)])
def test_direct_sum_matches_oracle(rbf, kernel, eps):
    import torch
    X, lam = workloads.uniform(5000, 3, 2)
    tg = np.arange(0, 5000, 37)
    ref = O.direct(X, lam, kernel, eps, tg)
    u = torch.empty(len(tg), dtype=torch.float64, device="cuda")
    rbf.direct_sum(_dev(X), kernel, eps, _dev(lam), _dev(tg.astype(np.int64)), u)
    assert rel(u.cpu().numpy(), ref) <= 1e-14


def test_direct_sum_out_of_range_targets_give_nan(rbf):
    """The kernel checks each target index: -1 and N read nothing and give NaN,
    the valid targets around them are unaffected."""
    import torch
    X, lam = workloads.uniform(3000, 2, 4)
    tg = np.array([5, -1, 17, 3000, 2999], dtype=np.int64)
    u = torch.empty(len(tg), dtype=torch.float64, device="cuda")
    rbf.direct_sum(_dev(X), O.IMQ, 2.0, _dev(lam), _dev(tg), u)
    got = u.cpu().numpy()
    assert np.isnan(got[1]) and np.isnan(got[3])
    ok = np.array([0, 2, 4])
    assert rel(got[ok], O.direct(X, lam, O.IMQ, 2.0, tg[ok])) <= 1e-14


def test_auto_box_and_bad_arguments(rbf):
    import torch
    X, lam = workloads.uniform(1000, 2, 5)
    X = X * 3.0 - 1.0
    t = rbf.tree_build(_dev(X), lo=None, depth=-1)
    info = t.info()
    assert np.allclose(info["lo"], X.min(axis=0))
    assert abs(info["side"] - np.max(X.max(axis=0) - X.min(axis=0))) < 1e-15
    u = torch.empty(1000, dtype=torch.float64, device="cuda")
    with pytest.raises(rbf.RbfError):
        rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), u, M=7)          # odd M
    with pytest.raises(rbf.RbfError):
        rbf.fmm_matvec(t, O.IMQ, -1.0, _dev(lam), u)              # eps <= 0
    with pytest.raises(rbf.RbfError):
        rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), u, M=16, period_L=1.5 * info["side"])  # L < 2 side with taper
    with pytest.raises(rbf.RbfError):
        rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), u, M=16, csample=0)  # closed form is Gaussian-only


@pytest.mark.parametrize("d,n,D,eps,kernel", [(3, 20000, 3, 77.0, O.GAUSSIAN),
                                              (2, 30000, 4, 120.0, O.GAUSSIAN),
                                              (3, 8000, 2, 4.5, O.WENDLAND)])
def test_near_field_only_product(rbf, d, n, D, eps, kernel):
    """M = 0: no far field.  The product is the oracle's near-field sum
    u_i = sum_{j in N(i)} lambda_j Phi(x_i - x_j) (FP64 <= 1e-12, FP32 <= 5e-6,
    element-wise too), and it is within max_far |Phi| * sum |lambda| of the
    direct sum (the Lemma bound of Eq. (33) with K = 0).  For these kernels
    Phi has fallen below 1e-15 at the nearest far offset (one leaf width), so
    the far field is exactly negligible; rbf_kernel_error reports that value."""
    import torch
    from paper_1606_07652_gb300 import _lib
    X, lam = workloads.uniform(n, d, seed=n + d)
    T = O.tree(X, np.zeros(d), 1.0, D)
    ls = lam[T["perm"]]
    near_sorted = O.p2p(T, ls, kernel, eps)
    ref = np.empty(n)
    ref[T["perm"]] = near_sorted
    t = rbf.tree_build(_dev(X), lo=np.zeros(d), side=1.0, depth=D)
    lam_d = _dev(lam)
    out = {}
    for prec in (rbf.FP64, rbf.FP32):
        u = torch.empty_like(lam_d)
        rbf.fmm_matvec(t, kernel, eps, lam_d, u, prec=prec, M=0)
        torch.cuda.synchronize()
        out[prec] = u.cpu().numpy()
    e64, e32 = rel(out[rbf.FP64], ref), rel(out[rbf.FP32], ref)
    print(f"near-field only d={d} eps={eps}: fp64 {e64:.2e} fp32 {e32:.2e}")
    assert e64 <= FP64_TOL and e32 <= FP32_TOL
    w = 1.0 / (1 << D)
    kerr = _lib.kernel_error(kernel, eps, d, 0, 4.0, 0.0, 1.0, D)
    assert kerr == pytest.approx(float(O.phi(kernel, eps, np.array([w]))[0]), rel=1e-12, abs=1e-300)
    assert kerr < 1e-15
    tg = np.arange(0, n, 97)
    ud = O.direct(X, lam, kernel, eps, tg)
    assert np.max(np.abs(out[rbf.FP64][tg] - ud)) <= kerr * np.sum(np.abs(lam)) + 1e-12 * np.max(np.abs(ud))


def test_autotune_picks_no_far_field_for_narrow_kernels(rbf):
    from paper_1606_07652_gb300 import _lib
    narrow = _lib.autotune(O.GAUSSIAN, 77.0, 3, 1 << 18, 1e-10)
    assert narrow["M"] == 0 and narrow["err"] <= 1e-10, narrow
    wide = _lib.autotune(O.GAUSSIAN, 3.0, 3, 1 << 18, 1e-8)
    assert wide["M"] >= 8, wide


def test_p2m_launch_shape_is_measured_and_bit_neutral(rbf):
    """An FP32 plan of a large enough tree times both P2M launch shapes when it is
    created and keeps the faster (rbf_p2m_launch_shape); a small tree keeps the rule.
    The shapes accumulate every output over the points in the same order, so two trees
    of the same points give the same bits whichever shape each picked (also with each
    shape forced through RBF_P2M_SHAPE), and the product matches the oracle's FMM."""
    import torch
    from paper_1606_07652_gb300 import _lib
    X, lam = workloads.uniform(20000, 3, 61)
    kw = dict(M=24, period_L=4.0, window_alpha=4.5)
    outs, shapes = [], []
    for _ in range(2):
        t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=3)
        u = torch.empty(len(X), dtype=torch.float64, device="cuda")
        rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), u, prec=rbf.FP32, **kw)
        torch.cuda.synchronize()
        shapes.append(_lib.p2m_launch_shape(t))
        outs.append(u.cpu().numpy())
        t.free()
    assert all(s in (1, 2) for s in shapes), shapes
    assert np.array_equal(outs[0], outs[1])
    # each shape forced in turn (dense, wide): the same bits
    forced = []
    old_env = os.environ.get("RBF_P2M_SHAPE")
    try:
        for shape in (1, 2):
            os.environ["RBF_P2M_SHAPE"] = str(shape)
            t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=3)
            u = torch.empty(len(X), dtype=torch.float64, device="cuda")
            rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), u, prec=rbf.FP32, **kw)
            torch.cuda.synchronize()
            assert _lib.p2m_launch_shape(t) == shape
            forced.append(u.cpu().numpy())
            t.free()
    finally:
        if old_env is None:
            os.environ.pop("RBF_P2M_SHAPE", None)
        else:
            os.environ["RBF_P2M_SHAPE"] = old_env
    for f in forced:
        assert np.array_equal(f, outs[0])
    T = O.tree(X, np.zeros(3), 1.0, 3)
    wc = O.coeffs_sampled(O.IMQ, 2.0, 3, 24, 4.0, 4.5, 1.0)
    assert rel(outs[0], O.fmm(T, lam, O.IMQ, 2.0, wc, 24, 4.0)) <= FP32_TOL
    Xs, lams = workloads.uniform(5000, 3, 62)
    ts = rbf.tree_build(_dev(Xs), lo=np.zeros(3), side=1.0, depth=3)
    us = torch.empty(len(Xs), dtype=torch.float64, device="cuda")
    rbf.fmm_matvec(ts, O.IMQ, 2.0, _dev(lams), us, prec=rbf.FP32, **kw)
    assert _lib.p2m_launch_shape(ts) == 0
    ts.free()
