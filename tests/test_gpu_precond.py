"""Learned approximate-cardinal preconditioner on the GPU against the oracle.

kNN lists are bit-exact; local cardinal coefficients match the FP64 oracle;
the BF16 tensor-core network matches the oracle network run with the same
BF16 operand rounding and FP64 sums (relative L2 <= 2e-2, the stated BF16
tolerance; the gap is FP32 against FP64 accumulation); training lowers the loss; the trained network's P cuts
GMRES iterations on a problem with local cardinal functions; on a flat kernel
the solve falls back to the plain iteration, judged by the FP64 residual."""
import numpy as np
import pytest

import oracle as O
from oracle.solver import bf16_round, cardinal, knn, mlp_backward, mlp_forward, mlp_init

pytestmark = pytest.mark.gpu

BF16_TOL = 2e-2


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1606_07652_gb300 as rbf
    from paper_1606_07652_gb300 import _lib
    rbf.load()
    return rbf, _lib, torch


def _dev(torch, a):
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def jittered(n1, seed):
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij"), -1).reshape(-1, 2)
    return (g + 0.5 + 0.3 * rng.uniform(-0.5, 0.5, (n1 * n1, 2))) / n1


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["uniform-3d", "clustered-2d", "lattice-ties"])
def test_knn_bit_exact(env, case):
    rbf, _lib, torch = env
    rng = np.random.default_rng(17)
    if case == "uniform-3d":
        X, D, d = rng.random((2000, 3)), 3, 3
    elif case == "clustered-2d":
        X = np.clip(rng.uniform(0.3, 0.7, (3, 2))[rng.integers(3, size=1500)]
                    + 0.02 * rng.standard_normal((1500, 2)), 0, 1)
        D, d = 5, 2
    else:  # exact lattice: many exactly equal distances, order decided by index
        g = np.stack(np.meshgrid(np.arange(20), np.arange(20), indexing="ij"), -1).reshape(-1, 2)
        X, D, d = (g + 0.5) / 32.0, 3, 2
    t = rbf.tree_build(_dev(torch, X), lo=np.zeros(d), side=1.0, depth=D)
    assert np.array_equal(_lib.knn(t), knn(X, 32))


def test_cardinal_matches_oracle(env):
    rbf, _lib, torch = env
    X = jittered(24, 5)
    t = rbf.tree_build(_dev(torch, X), lo=np.zeros(2), side=1.0, depth=3)
    centres = np.arange(0, len(X), 7)
    c = _lib.cardinal_weights(t, rbf.GAUSSIAN, 28.8, 1e-12, centres)
    ref = cardinal(X, knn(X, 32)[centres], O.GAUSSIAN, 28.8, 1e-12)
    assert rel(c, ref) <= 1e-9


def _oracle_params(W, b):
    return np.concatenate([np.concatenate([Wl.ravel(), bl]) for Wl, bl in zip(W, b)])


def test_mlp_forward_and_gradient_match_oracle(env):
    rbf, _lib, torch = env
    rng = np.random.default_rng(9)
    W, b = mlp_init([64, 128, 128, 128, 32], seed=4)
    for bl in b:
        bl += 0.05 * rng.standard_normal(bl.shape)
    X = rng.standard_normal((300, 64)) * 0.5
    T = rng.standard_normal((300, 32)) * 0.1
    net = _lib.Mlp(64, 128, 32, seed=1)
    net.set_params(_oracle_params(W, b).astype(np.float32))
    Xd = _dev(torch, X.astype(np.float32))
    Y = torch.empty((300, 32), dtype=torch.float32, device="cuda")
    net.forward(Xd, Y)
    G = torch.empty(net.num_params(), dtype=torch.float32, device="cuda")
    loss = net.gradient(Xd, _dev(torch, T.astype(np.float32)), G)
    torch.cuda.synchronize()
    # oracle with the BF16 operand rounding of every product (FP64 sums), so that both
    # sides take the ReLU decisions from the same operands
    Yo, cache = mlp_forward(W, b, X, q=bf16_round)
    gW, gb = mlp_backward(W, b, cache, Yo, T, q=bf16_round)
    assert rel(Y.cpu().numpy(), Yo) <= BF16_TOL
    assert abs(loss - np.mean((Yo - T) ** 2)) <= BF16_TOL * np.mean((Yo - T) ** 2)
    g = G.cpu().numpy()
    assert rel(g, _oracle_params(gW, gb)) <= BF16_TOL
    for l in range(4):   # every layer, not only the largest
        off = sum(W[q].size + b[q].size for q in range(l))
        assert rel(g[off:off + W[l].size], gW[l].ravel()) <= BF16_TOL


def test_training_and_learned_preconditioner_gain(env):
    """Trained on a 64 x 64 jittered grid, applied to a 24 x 24 one at the same
    eps*h = 1.2 (the features eps (x_j - x_i) do not depend on the grid size): the
    learned P cuts GMRES iterations against the plain solve (local cardinal
    functions are local in this regime)."""
    rbf, _lib, torch = env
    eps, M, L, D = 28.8, 64, 1.208, 3
    kw = dict(M=M, period_L=L, window_alpha=0.0)
    Xa = jittered(64, 11)
    ta = rbf.tree_build(_dev(torch, Xa), lo=np.zeros(2), side=1.0, depth=4)
    net = _lib.Mlp(64, 128, 32, seed=7)
    rep = _lib.precond_train(ta, rbf.GAUSSIAN, 1.2 * 64, net, n_train=4096, epochs=300, batch=512,
                             lr=1e-3, delta_rel=1e-12)
    assert rep["loss_last"] < 1e-2 * rep["loss_first"], rep
    Xb = jittered(24, 12)
    tb = rbf.tree_build(_dev(torch, Xb), lo=np.zeros(2), side=1.0, depth=D)
    u = np.sin(2 * np.pi * Xb[:, 0]) * np.cos(2 * np.pi * Xb[:, 1])
    ud = _dev(torch, u)
    lam0 = torch.zeros_like(ud)
    plain = rbf.interp_solve(tb, rbf.GAUSSIAN, eps, ud, lam0, rtol=1e-9, inner_prec=rbf.FP64,
                             precond=0, **kw)
    _lib.precond_build(tb, rbf.GAUSSIAN, eps, net)
    lam1 = torch.zeros_like(ud)
    learned = rbf.interp_solve(tb, rbf.GAUSSIAN, eps, ud, lam1, rtol=1e-9, inner_prec=rbf.FP64,
                               precond=1, **kw)
    _lib.precond_build(tb, rbf.GAUSSIAN, eps, None)
    lam2 = torch.zeros_like(ud)
    exact = rbf.interp_solve(tb, rbf.GAUSSIAN, eps, ud, lam2, rtol=1e-9, inner_prec=rbf.FP64,
                             precond=1, **kw)
    print("iterations plain", plain["iters"], "learned", learned["iters"], "exact local",
          exact["iters"])
    for r in (plain, learned, exact):
        assert r["status"] == 0 and r["rel_resid"] <= 1e-9, r
    assert learned["used_fallback"] == 0
    assert learned["iters"] < plain["iters"]
    assert exact["iters"] < plain["iters"]
    # the preconditioned solution solves the same system (oracle FMM residual)
    T = O.tree(Xb, np.zeros(2), 1.0, D)
    wc = O.coeffs_sampled(O.GAUSSIAN, eps, 2, M, L, 0.0, 1.0)
    res = rel(O.fmm(T, lam1.cpu().numpy(), O.GAUSSIAN, eps, wc, M, L), u)
    assert res <= 1.5e-9


def test_flat_kernel_falls_back(env):
    """Gaussian eps*h = 0.25: local cardinal functions are not local and the
    preconditioned step does not lower the FP64 residual; the solve drops P."""
    rbf, _lib, torch = env
    eps, M, L, D = 6.0, 32, 2.5, 3
    kw = dict(M=M, period_L=L, window_alpha=0.0)
    X = jittered(24, 13)
    t = rbf.tree_build(_dev(torch, X), lo=np.zeros(2), side=1.0, depth=D)
    _lib.precond_build(t, rbf.GAUSSIAN, eps, None)
    u = np.sin(2 * np.pi * X[:, 0]) * np.cos(2 * np.pi * X[:, 1])
    ud = _dev(torch, u)
    lam = torch.zeros_like(ud)
    rep = rbf.interp_solve(t, rbf.GAUSSIAN, eps, ud, lam, rtol=1e-12, restart_m=30, max_iters=300,
                           max_refine=6, inner_prec=rbf.FP64, precond=1, **kw)
    print(rep)
    assert rep["used_fallback"] == 1
    assert np.all(np.isfinite(lam.cpu().numpy()))


def test_precond_apply_matches_oracle(env):
    rbf, _lib, torch = env
    X = jittered(24, 14)
    eps = 28.8
    t = rbf.tree_build(_dev(torch, X), lo=np.zeros(2), side=1.0, depth=3)
    _lib.precond_build(t, rbf.GAUSSIAN, eps, None, delta_rel=1e-12)
    y = np.random.default_rng(2).standard_normal(len(X))
    z = torch.empty(len(X), dtype=torch.float64, device="cuda")
    _lib.precond_apply(t, _dev(torch, y), z)
    nb = knn(X, 32)
    c = cardinal(X, nb, O.GAUSSIAN, eps, 1e-12)
    A = O.phi(O.GAUSSIAN, eps, np.linalg.norm(X[:, None] - X[None], axis=2))
    zr = np.zeros(len(X))
    for i in range(len(X)):
        w = c[i] / (A[i, nb[i]] @ c[i])
        zr[nb[i]] += w * y[i]
    assert rel(z.cpu().numpy(), zr) <= 1e-9


def test_network_checkpoint_resumes_training_exactly(env, tmp_path):
    """rbf_mlp_save / rbf_mlp_load: the reloaded network has the same parameters and
    Adam state, so further steps give the same losses and parameters bit for bit;
    truncated and foreign files are rejected."""
    rbf, _lib, torch = env
    rng = np.random.default_rng(8)
    X = torch.as_tensor(rng.standard_normal((256, 96)).astype(np.float32), device="cuda")
    T = torch.as_tensor(rng.standard_normal((256, 32)).astype(np.float32), device="cuda")
    a = _lib.Mlp(96, 128, 32, seed=3)
    for _ in range(5):
        a.train_step(X, T, 1e-3)
    path = str(tmp_path / "net.bin")
    a.save(path)
    b = _lib.Mlp.load_checkpoint(path)
    assert (b.d_in, b.width, b.d_out) == (96, 128, 32)
    assert np.array_equal(a.get_params(), b.get_params())
    la = [a.train_step(X, T, 1e-3) for _ in range(3)]
    lb = [b.train_step(X, T, 1e-3) for _ in range(3)]
    assert la == lb
    assert np.array_equal(a.get_params(), b.get_params())
    raw = open(path, "rb").read()
    bad = tmp_path / "short.bin"
    bad.write_bytes(raw[: len(raw) // 2])
    with pytest.raises(rbf.RbfError) as e:
        _lib.Mlp.load_checkpoint(str(bad))
    assert e.value.code == -1
    foreign = tmp_path / "foreign.bin"
    foreign.write_bytes(b"NOTANMLP" + raw[8:])
    with pytest.raises(rbf.RbfError):
        _lib.Mlp.load_checkpoint(str(foreign))
