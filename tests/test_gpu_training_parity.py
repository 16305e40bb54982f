"""Parity of the learned preconditioner's input features and optimiser step.

* Features: rbf_precond_features writes eps (x_j - x_i) for the 32 nearest
  neighbours j of each requested centre i, nearest first, in FP32.  Both sides
  form the difference and the product in FP64 and round once, so the GPU rows
  equal the oracle's ``features`` rounded to FP32 bit for bit.
* Adam: rbf_mlp_train_step = the gradient of rbf_mlp_gradient (the same
  deterministic kernels at the same weights) followed by one Adam update
  (Kingma & Ba; beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected moments) of
  the FP32 master weights.  Feeding the GPU's gradients to the oracle's
  ``adam_step`` in FP64 reproduces the GPU weights after three steps to within
  FP32 rounding of the weights (bound 1e-6 absolute; a dropped bias correction
  or moment changes them by about the learning rate, 1e-3).
"""
import numpy as np
import pytest

from oracle.solver import adam_step, features, knn

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


@pytest.mark.parametrize("d", [2, 3])
def test_features_bit_exact(env, d):
    rbf, _lib, torch = env
    rng = np.random.default_rng(40 + d)
    X = rng.random((600, d))
    eps = 7.5
    t = rbf.tree_build(torch.as_tensor(X, device="cuda"), lo=np.zeros(d), side=1.0, depth=2)
    centres = np.array([0, 1, 17, 299, 598, 599, 333, 17], dtype=np.int64)   # repeats allowed
    F = torch.empty((len(centres), 32 * d), dtype=torch.float32, device="cuda")
    _lib.precond_features(t, eps, centres, F)
    torch.cuda.synchronize()
    ref = features(X, knn(X, 32), eps)[centres].astype(np.float32)
    assert np.array_equal(F.cpu().numpy(), ref)


def test_adam_steps_match_oracle(env):
    rbf, _lib, torch = env
    rng = np.random.default_rng(12)
    X = torch.as_tensor(rng.standard_normal((200, 64)).astype(np.float32), device="cuda")
    T = torch.as_tensor(0.1 * rng.standard_normal((200, 32)).astype(np.float32), device="cuda")
    net = _lib.Mlp(64, 128, 32, seed=9)
    lr = 1e-3
    p0 = net.get_params().astype(np.float64)
    p = p0.copy()
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    G = torch.empty(net.num_params(), dtype=torch.float32, device="cuda")
    for step in (1, 2, 3):
        net.gradient(X, T, G)
        g = G.cpu().numpy().astype(np.float64)
        net.train_step(X, T, lr)
        adam_step(p, g, m, v, step, lr)
        got = net.get_params().astype(np.float64)
        err = float(np.max(np.abs(got - p)))
        print(f"step {step}: max |w_gpu - w_oracle| = {err:.2e}")
        assert err <= 1e-6
    # three steps moved the typical weight by the order of the learning rate
    assert float(np.median(np.abs(got - p0))) > 0.1 * lr
