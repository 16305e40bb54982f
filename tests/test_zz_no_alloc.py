"""The allocation-free Morton ordering entry point against the regular tree build.

rbf_morton_order_noalloc serves callers that must not allocate device memory
at call time (a framework's pool already owns the free memory, or a step loop
cannot afford cudaMalloc/cudaFree latency and device synchronisation).  It
keeps its temporaries in a fixed device arena shared by all calls, so the
test runs it twice in a row on different inputs and requires each result to
equal, bit for bit, the keys and permutation that rbf_tree_build stores.
This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_07652_gb300 as rbf
    from paper_1606_07652_gb300 import _lib
    rbf.load()
    return rbf, _lib, torch


def _reference(rbf, torch, X, d, depth):
    t = rbf.tree_build(torch.as_tensor(X, device="cuda"), lo=np.zeros(d), side=1.0, depth=depth)
    e = t.export()
    t.free()
    return e["perm"], e["keys"]


def _noalloc(_lib, torch, X, d, depth):
    Xd = torch.as_tensor(X, device="cuda")
    perm = torch.full((len(X),), -1, dtype=torch.int32, device="cuda")
    keys = torch.zeros(len(X), dtype=torch.int64, device="cuda")
    _lib.morton_order_noalloc(Xd, np.zeros(d), 1.0, depth, perm, keys)
    torch.cuda.synchronize()
    return perm.cpu().numpy().astype(np.int64), keys.cpu().numpy().view(np.uint64)


def test_two_calls_match_tree_build(env):
    rbf, _lib, torch = env
    X1, _ = workloads.uniform(300001, 3, 41)           # 18 key bits: three digit passes
    rng = np.random.default_rng(42)
    X2 = np.clip(rng.uniform(0.3, 0.7, (4, 2))[rng.integers(4, size=70000)]
                 + 0.02 * rng.standard_normal((70000, 2)), 0, 1)   # clustered, two passes
    for X, d, depth in ((X1, 3, 6), (X2, 2, 7)):
        perm, keys = _noalloc(_lib, torch, X, d, depth)
        ref_perm, ref_keys = _reference(rbf, torch, X, d, depth)
        assert np.array_equal(perm, ref_perm)
        assert np.array_equal(keys, ref_keys)


def test_depth_zero_and_single_centre(env):
    """No radix pass runs when there are no key bits (depth 0) or one centre:
    the keys and the identity order then come straight from the key kernel."""
    rbf, _lib, torch = env
    X0, _ = workloads.uniform(5000, 3, 43)
    X1 = np.array([[0.25, 0.75, 0.5]])
    X1b = np.array([[0.9, 0.1]])
    for X, d, depth in ((X0, 3, 0), (X1, 3, 4), (X1b, 2, 0), (X0, 3, 0)):
        perm, keys = _noalloc(_lib, torch, X, d, depth)
        ref_perm, ref_keys = _reference(rbf, torch, X, d, depth)
        assert np.array_equal(perm, ref_perm)
        assert np.array_equal(keys, ref_keys)


def test_size_limit_is_rejected(env):
    rbf, _lib, torch = env
    X = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    perm = torch.zeros(4, dtype=torch.int32, device="cuda")
    keys = torch.zeros(4, dtype=torch.int64, device="cuda")
    lo = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    code = _lib.load().rbf_morton_order_noalloc(ctypes.c_void_p(X.data_ptr()), (1 << 22) + 1, 3,
                                                lo, 1.0, 5, ctypes.c_void_p(perm.data_ptr()),
                                                ctypes.c_void_p(keys.data_ptr()), None)
    assert code == -1
    assert b"arena" in _lib.load().rbf_last_error()
