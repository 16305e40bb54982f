"""GPU parity of the evaluation at new points (rbf_eval_create / rbf_eval_apply).

s(y) = sum_j lambda_j Phi(y - x_j) at points y that are not centres, through one
tree over the centres and the new points.  Compared element by element with the
oracle's evaluation on the same inputs (FP64 1e-12, FP32 5e-6), for several
kernels, dimensions and columns; new points outside the root cube are
rejected; at N = 2^20 the evaluation is checked against the direct sum.
"""
import numpy as np
import pytest

import oracle as O
import workloads
from _parity import rel

pytestmark = pytest.mark.gpu


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


CASES = [
    # name, d, N, nt, D, kernel, eps, M, L, alpha, nrhs
    ("2d-imq", 2, 5000, 2000, 4, O.IMQ, 2.0, 16, 4.0, 4.5, 1),
    ("3d-gauss-3cols", 3, 6000, 1500, 3, O.GAUSSIAN, 3.0, 12, 3.0, 0.0, 3),
    ("2d-mq", 2, 3000, 3000, 3, O.MQ, 1.0, 20, 4.0, 4.5, 1),
    ("1d-wendland", 1, 2000, 700, 4, O.WENDLAND, 0.5, 16, 4.0, 0.0, 2),
    ("3d-imq-5cols", 3, 8000, 4000, 3, O.IMQ, 2.0, 16, 4.0, 4.5, 5),
]


@pytest.mark.parametrize("name,d,n,nt,D,kernel,eps,M,L,alpha,nrhs", CASES)
def test_evaluate_matches_oracle(rbf, name, d, n, nt, D, kernel, eps, M, L, alpha, nrhs):
    import torch
    X, _ = workloads.uniform(n, d, seed=n + d)
    Y = np.random.default_rng(n + nt).random((nt, d))
    lam = np.random.default_rng(nt).standard_normal((nrhs, n))
    wc = O.coeffs_sampled(kernel, eps, d, M, L, alpha, 1.0)
    t = rbf.tree_build(_dev(X), lo=np.zeros(d), side=1.0, depth=D)
    ev = rbf.Evaluator(t, _dev(Y))
    kw = dict(M=M, period_L=L, window_alpha=alpha)
    out = {}
    for prec in (rbf.FP64, rbf.FP32):
        S = torch.empty((nrhs, nt), dtype=torch.float64, device="cuda")
        ev.apply(kernel, eps, _dev(lam), S, prec=prec, **kw)
        torch.cuda.synchronize()
        out[prec] = S.cpu().numpy()
    for c in range(nrhs):
        ref = O.fmm_evaluate(X, lam[c], Y, np.zeros(d), 1.0, D, kernel, eps, wc, M, L)
        e64, e32 = rel(out[rbf.FP64][c], ref), rel(out[rbf.FP32][c], ref)
        print(f"{name} col {c}: FP64 {e64:.2e}, FP32 {e32:.2e}")
        assert e64 <= 1e-12
        assert e32 <= 5e-6
    ev.free()


def test_evaluate_rejects_points_outside_the_root(rbf):
    X, _ = workloads.uniform(1000, 2, 3)
    t = rbf.tree_build(_dev(X), lo=np.zeros(2), side=1.0, depth=3)
    Y = np.array([[0.5, 0.5], [1.2, 0.3]])
    with pytest.raises(rbf.RbfError) as e:
        rbf.Evaluator(t, _dev(Y))
    assert e.value.code == -1


def test_evaluate_full_size_3d(rbf):
    """N = 2^20 centres (IMQ eps = 2, depth 5, M = 32), 2^16 new points: the FP32
    evaluation matches the FP64 evaluation to the FP32 bound, and its error
    against the direct sum on 1024 of the new points is within 2x of the
    product's own error at the centres."""
    import torch
    X, lam, targets, p = workloads.config2()
    Y = np.random.default_rng(99).random((1 << 16, 3))
    t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=p["depth"])
    ev = rbf.Evaluator(t, _dev(Y))
    kw = dict(M=p["M"], period_L=p["L"], window_alpha=p["alpha"])
    ld = _dev(lam)
    s32 = torch.empty(len(Y), dtype=torch.float64, device="cuda")
    s64 = torch.empty_like(s32)
    ev.apply(p["kernel"], p["eps"], ld, s32, prec=rbf.FP32, **kw)
    ev.apply(p["kernel"], p["eps"], ld, s64, prec=rbf.FP64, **kw)
    u = torch.empty_like(ld)
    rbf.fmm_matvec(t, p["kernel"], p["eps"], ld, u, prec=rbf.FP32, **kw)
    torch.cuda.synchronize()
    assert rel(s32.cpu().numpy(), s64.cpu().numpy()) < 5e-6
    pick = np.random.default_rng(5).choice(len(Y), 1024, replace=False)
    Z = np.concatenate([X, Y[pick]])
    sd = O.direct(Z, np.concatenate([lam, np.zeros(1024)]), p["kernel"], p["eps"],
                  np.arange(len(X), len(Z)))
    ud = O.direct(X, lam, p["kernel"], p["eps"], targets[:1024])
    e_eval = rel(s32.cpu().numpy()[pick], sd)
    e_prod = rel(u.cpu().numpy()[targets[:1024]], ud)
    print(f"N=2^20, 2^16 new points: evaluation {e_eval:.2e}, product {e_prod:.2e} vs direct")
    assert e_eval <= 2.0 * e_prod + 1e-7
    ev.free()
