"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The oracle cannot run the whole multilevel FMM at N = 2^20, so it computes sampled
outputs one by one from the definition of what the FMM computes,
    u_i = sum_{j near} lambda_j Phi(x_i - x_j) + sum_{j far} lambda_j K(x_i - x_j)
(oracle.fmm_at_targets, pinned against the oracle's multilevel FMM in
test_oracle_pins.py).  The samples reach leaves of every occupancy (first and
last point of each), every point of the most crowded leaf and leaves on the
root cube's boundary, and each is bounded element by element.  At every size the FP64 product must also satisfy the
far-field bound of the scaled Lemma, Eq. (33), against the direct sum."""
import numpy as np
import pytest

import oracle as O
import workloads
from _parity import errs, spread_sample

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_07652_gb300 as rbf
    rbf.load()
    return rbf, torch


def _gpu_products(rbf, torch, X, lam, depth, p):
    t = rbf.tree_build(torch.as_tensor(X, device="cuda"), lo=np.zeros(X.shape[1]), side=1.0,
                       depth=depth)
    ld = torch.as_tensor(lam, device="cuda")
    kw = dict(M=p["M"], period_L=p["L"], window_alpha=p["alpha"])
    u64 = torch.empty_like(ld)
    u32 = torch.empty_like(ld)
    rbf.fmm_matvec(t, p["kernel"], p["eps"], ld, u64, prec=rbf.FP64, **kw)
    rbf.fmm_matvec(t, p["kernel"], p["eps"], ld, u32, prec=rbf.FP32, **kw)
    torch.cuda.synchronize()
    return t, ld, u64.cpu().numpy(), u32.cpu().numpy()


def test_bench_workload_sampled_parity_and_lemma_bound(env):
    """3-D, N = 2^20 uniform, IMQ eps = 2, depth 5, M = 32, L = 4, alpha = 4.5 (bench.py)."""
    rbf, torch = env
    X, lam, targets, p = workloads.config2()
    t, ld, u64, u32 = _gpu_products(rbf, torch, X, lam, p["depth"], p)
    T = O.tree(X, np.zeros(3), 1.0, p["depth"])
    wc = O.coeffs_sampled(p["kernel"], p["eps"], 3, p["M"], p["L"], p["alpha"], 1.0)
    rng = np.random.default_rng(20)
    sorted_pick = spread_sample(T["leaf_off"], rng, keys=T["leaf_key"], d=3, depth=p["depth"])
    assert len(sorted_pick) >= 256
    sample = T["perm"][sorted_pick]
    ref = O.fmm_at_targets(T, lam, p["kernel"], p["eps"], wc, p["M"], p["L"], sample)
    e64, e32 = errs(u64[sample], ref), errs(u32[sample], ref)
    print(f"N=2^20 sampled parity on {len(sample)} targets (leaf sizes "
          f"{np.diff(T['leaf_off']).min()}..{np.diff(T['leaf_off']).max()}): "
          f"fp64 rel-L2 {e64[0]:.2e} max {e64[1]:.2e}  fp32 rel-L2 {e32[0]:.2e} max {e32[1]:.2e}")
    assert max(e64) <= 1e-12
    assert max(e32) <= 5e-6
    # Lemma (33): |u_fmm - u_direct|_i <= max_far |K - Phi| * sum_j |lambda_j|, on 4096 targets
    tg = torch.as_tensor(np.asarray(targets, dtype=np.int64), device="cuda")
    ud = torch.empty(len(targets), dtype=torch.float64, device="cuda")
    rbf.direct_sum(torch.as_tensor(X, device="cuda"), p["kernel"], p["eps"], ld, tg, ud)
    ud = ud.cpu().numpy()
    rng = np.random.default_rng(21)
    r = rng.uniform(-1, 1, (3000, 3))
    r = r[np.max(np.abs(r), axis=1) >= 1.0 / 32]
    kerr = np.max(np.abs(O.kernel_K(wc, 3, p["M"], p["L"], r)
                         - O.phi(p["kernel"], p["eps"], np.linalg.norm(r, axis=1))))
    bound = kerr * np.sum(np.abs(lam))
    assert np.max(np.abs(u64[targets] - ud)) <= bound


def test_clustered_workload_sampled_parity(env):
    """3-D, N = 262,144 clustered (8 Gaussians), Gaussian eps = 3, depth 6, M = 24, L = 3:
    leaves range from empty to ~90 points."""
    rbf, torch = env
    X, u, p = workloads.config3()
    lam = np.random.default_rng(77).standard_normal(len(X))
    t, ld, u64, u32 = _gpu_products(rbf, torch, X, lam, 6, p)
    T = O.tree(X, np.zeros(3), 1.0, 6)
    wc = O.coeffs_sampled(p["kernel"], p["eps"], 3, p["M"], p["L"], p["alpha"], 1.0)
    rng = np.random.default_rng(78)
    sorted_pick = spread_sample(T["leaf_off"], rng, keys=T["leaf_key"], d=3, depth=6)
    assert len(sorted_pick) >= 256
    sample = T["perm"][sorted_pick]
    ref = O.fmm_at_targets(T, lam, p["kernel"], p["eps"], wc, p["M"], p["L"], sample)
    e64, e32 = errs(u64[sample], ref), errs(u32[sample], ref)
    print(f"clustered sampled parity on {len(sample)} targets (leaf sizes "
          f"{np.diff(T['leaf_off']).min()}..{np.diff(T['leaf_off']).max()}): "
          f"fp64 rel-L2 {e64[0]:.2e} max {e64[1]:.2e}  fp32 rel-L2 {e32[0]:.2e} max {e32[1]:.2e}")
    assert max(e64) <= 1e-12
    assert max(e32) <= 5e-6


def test_fp32_telescoped_coupling_does_not_degrade_with_n(env):
    """The shared-grid coupling forms every leaf's local expansion as the root
    expansion, translated, minus the near leaves' terms (telescoped M2L + L2L).
    In FP32 that difference could lose digits as the root sum grows with N.  At
    fixed depth (5) and M = 32 the FP32 product is compared element by element with
    the FP64 product (itself pinned to the oracle at 1e-12) at N = 2^18, 2^20 and
    2^22 (8 to 128 points per leaf): every element within 5e-6 of max |u|, and the
    error at 2^22 no more than 4x the error at 2^18 (a cancellation that grew with
    N would give 16x for a 16x larger root sum)."""
    rbf, torch = env
    p = dict(kernel=O.IMQ, eps=2.0, M=32, L=4.0, alpha=4.5)
    worst = {}
    for n in (1 << 18, 1 << 20, 1 << 22):
        X, lam = workloads.uniform(n, 3, 90 + n % 7)
        t, ld, u64, u32 = _gpu_products(rbf, torch, X, lam, 5, p)
        e = errs(u32, u64)
        worst[n] = e[1]
        print(f"N={n}: fp32 vs fp64 rel-L2 {e[0]:.2e} max {e[1]:.2e} of max |u|")
        assert max(e) <= 5e-6
        t.free()
        del ld
        torch.cuda.empty_cache()
    assert worst[1 << 22] <= 4.0 * worst[1 << 18] + 1e-7
