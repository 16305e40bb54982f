"""Unwritten entries: with RBF_POISON set, every device allocation of the
library starts as all-ones bytes (NaN in FP32 and FP64).  Products on fresh
trees (so that every plan, expansion array, workspace and table is a new,
poisoned allocation) must still match the oracle: an entry read before it is
written would turn the result into NaN."""
import os

import numpy as np
import pytest

import oracle as O
import workloads
from _parity import rel
from oracle import nested as ON

pytestmark = pytest.mark.gpu


@pytest.fixture()
def rbf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_07652_gb300 as m
    m.load()
    os.environ["RBF_POISON"] = "1"
    yield m
    del os.environ["RBF_POISON"]


def _dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def test_poisoned_single_and_multi_column(rbf):
    import torch
    X, _ = workloads.uniform(7000, 3, 71)
    lam = np.random.default_rng(72).standard_normal((6, len(X)))
    T = O.tree(X, np.zeros(3), 1.0, 3)
    wc = O.coeffs_sampled(O.IMQ, 2.0, 3, 12, 4.0, 4.5, 1.0)
    t = rbf.tree_build(_dev(X), lo=np.zeros(3), side=1.0, depth=3)
    kw = dict(M=12, period_L=4.0, window_alpha=4.5)
    ref = [O.fmm(T, lam[c], O.IMQ, 2.0, wc, 12, 4.0) for c in range(6)]
    for prec, tol in ((rbf.FP64, 1e-12), (rbf.FP32, 5e-6)):
        u = torch.full((len(X),), float("nan"), dtype=torch.float64, device="cuda")
        rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam[0]), u, prec=prec, **kw)
        U = torch.full((6, len(X)), float("nan"), dtype=torch.float64, device="cuda")
        rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), U, prec=prec, **kw)
        torch.cuda.synchronize()
        assert torch.isfinite(u).all() and torch.isfinite(U).all()
        assert rel(u.cpu().numpy(), ref[0]) <= tol
        for c in range(6):
            assert rel(U[c].cpu().numpy(), ref[c]) <= tol


def test_poisoned_tensor_core_block(rbf):
    import torch
    X, _, p = workloads.config1()
    lam = np.random.default_rng(73).standard_normal((5, len(X)))
    T = O.tree(X, np.zeros(2), 1.0, 2)
    wc = O.coeffs_sampled(p["kernel"], p["eps"], 2, p["M"], p["L"], p["alpha"], 1.0)
    t = rbf.tree_build(_dev(X), lo=np.zeros(2), side=1.0, depth=2)
    U = torch.full((5, len(X)), float("nan"), dtype=torch.float64, device="cuda")
    rbf.fmm_matvec(t, p["kernel"], p["eps"], _dev(lam), U, prec=rbf.FP32, M=p["M"],
                   period_L=p["L"], window_alpha=p["alpha"])
    torch.cuda.synchronize()
    rbf.check_device_waits()
    for c in range(5):
        assert rel(U[c].cpu().numpy(), O.fmm(T, lam[c], p["kernel"], p["eps"], wc, p["M"], p["L"])) <= 5e-6


def test_poisoned_nested_and_evaluation(rbf):
    import torch
    X, lam = workloads.uniform(5000, 2, 74)
    T = O.tree(X, np.zeros(2), 1.0, 4)
    wcs = ON.coeffs_levels(O.IMQ, 2.0, 2, 16, 4.0, 4.5, 1.0, 4)
    t = rbf.tree_build(_dev(X), lo=np.zeros(2), side=1.0, depth=4)
    u = torch.full((len(X),), float("nan"), dtype=torch.float64, device="cuda")
    rbf.fmm_matvec(t, O.IMQ, 2.0, _dev(lam), u, prec=rbf.FP64, M=16, period_L=4.0, window_alpha=4.5,
                   grid=rbf.GRID_NESTED, lagrange_K=8)
    torch.cuda.synchronize()
    assert rel(u.cpu().numpy(), ON.fmm(T, lam, O.IMQ, 2.0, wcs, 16, 4.0, 8)) <= 1e-12
    Y = np.random.default_rng(75).random((900, 2))
    wc = O.coeffs_sampled(O.IMQ, 2.0, 2, 16, 4.0, 4.5, 1.0)
    ev = rbf.Evaluator(t, _dev(Y))
    s = torch.full((900,), float("nan"), dtype=torch.float64, device="cuda")
    ev.apply(O.IMQ, 2.0, _dev(lam), s, prec=rbf.FP64, M=16, period_L=4.0, window_alpha=4.5)
    torch.cuda.synchronize()
    ref = O.fmm_evaluate(X, lam, Y, np.zeros(2), 1.0, 4, O.IMQ, 2.0, wc, 16, 4.0)
    assert rel(s.cpu().numpy(), ref) <= 1e-12
    ev.free()
