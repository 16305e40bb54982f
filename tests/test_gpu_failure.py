"""Failure detection on the GPU without a fault: a bounded wait on an mbarrier
that nothing completes gives up within its limit, the kernel returns, the host
reads RBF_ETIMEOUT once, and the context stays usable for the next product."""
import numpy as np
import pytest

import oracle as O
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rbf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_07652_gb300 as m
    m.load()
    return m


def test_bounded_wait_gives_up_and_reports(rbf):
    import time
    import torch
    from paper_1606_07652_gb300 import _lib
    rbf.check_device_waits()                   # clean start
    t0 = time.perf_counter()
    assert _lib.selftest_bounded_wait(0.05) == 1
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(rbf.RbfError) as e:
        rbf.check_device_waits()
    assert e.value.code == -5
    rbf.check_device_waits()                   # the status was read and cleared
    # the context still computes: a four-column product through the tensor cores
    X, lam, p = workloads.config1()
    lam4 = np.random.default_rng(3).standard_normal((4, len(X)))
    t = rbf.tree_build(torch.as_tensor(X, device="cuda"), lo=np.zeros(2), side=1.0, depth=2)
    U = torch.empty((4, len(X)), dtype=torch.float64, device="cuda")
    rbf.fmm_matvec(t, p["kernel"], p["eps"], torch.as_tensor(lam4, device="cuda"), U, prec=rbf.FP32,
                   M=p["M"], period_L=p["L"], window_alpha=p["alpha"])
    torch.cuda.synchronize()
    rbf.check_device_waits()
    T = O.tree(X, np.zeros(2), 1.0, 2)
    wc = O.coeffs_sampled(p["kernel"], p["eps"], 2, p["M"], p["L"], p["alpha"], 1.0)
    ref = O.fmm(T, lam4[3], p["kernel"], p["eps"], wc, p["M"], p["L"])
    assert np.linalg.norm(U[3].cpu().numpy() - ref) / np.linalg.norm(ref) < 5e-6


def test_selftest_rejects_bad_limits(rbf):
    from paper_1606_07652_gb300 import _lib
    for s in (0.0, -1.0, 3.0):
        with pytest.raises(rbf.RbfError) as e:
            _lib.selftest_bounded_wait(s)
        assert e.value.code == -1
