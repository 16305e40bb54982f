"""Shape checks of the Python binding (host logic, no GPU).

The C entry points take raw device pointers and sizes and cannot see how large
a buffer is, so the binding checks every tensor's shape before it calls the
library: a too-short output, a block with the wrong number of columns or rows,
or a network input of the wrong width raises ValueError and nothing is
written.  These tests use CPU tensors and a stand-in tree: a call whose shapes
are right gets past the checks and stops at the device-tensor check
(TypeError), a call whose shapes are wrong stops at the shape check
(ValueError).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1606_07652_gb300 import _lib  # noqa: E402


class FakeTree:
    """Answers info() like a tree of N centres in d dimensions."""

    def __init__(self, N, d):
        self._info = {"N": N, "d": d, "side": 1.0}
        self.handle = None

    def info(self):
        return dict(self._info)


def f64(*shape):
    return torch.zeros(shape, dtype=torch.float64)


def test_helpers():
    assert _lib._rows_cols(f64(7), "a") == (1, 7)
    assert _lib._rows_cols(f64(3, 7), "a") == (3, 7)
    with pytest.raises(ValueError):
        _lib._rows_cols(f64(2, 3, 7), "a")
    _lib._expect(f64(3, 7), (3, 7), "a")
    with pytest.raises(ValueError):
        _lib._expect(f64(3, 6), (3, 7), "a")
    assert _lib._block(7, f64(3, 7), f64(3, 7), ("lam", "u")) == 3
    with pytest.raises(ValueError):
        _lib._block(7, f64(3, 6), f64(3, 6), ("lam", "u"))     # columns of the wrong length
    with pytest.raises(ValueError):
        _lib._block(7, f64(3, 7), f64(2, 7), ("lam", "u"))     # fewer output rows
    with pytest.raises(ValueError):
        _lib._block(7, f64(7), f64(6), ("lam", "u"))           # short output


def test_fmm_matvec_shapes():
    t = FakeTree(100, 3)
    with pytest.raises(TypeError):                              # shapes fine: device check next
        _lib.fmm_matvec(t, _lib.IMQ, 2.0, f64(100), f64(100), M=8)
    with pytest.raises(TypeError):
        _lib.fmm_matvec(t, _lib.IMQ, 2.0, f64(4, 100), f64(4, 100), M=8)
    for lam, u in ((f64(100), f64(99)), (f64(99), f64(99)), (f64(4, 100), f64(3, 100)),
                   (f64(4, 100), f64(100)), (f64(2, 2, 100), f64(2, 2, 100))):
        with pytest.raises(ValueError):
            _lib.fmm_matvec(t, _lib.IMQ, 2.0, lam, u, M=8)


def test_host_matvec_and_solve_shapes():
    t = FakeTree(50, 2)
    with pytest.raises(ValueError):
        _lib.fmm_matvec_host(t, _lib.IMQ, 2.0, np.zeros(50), np.zeros(49), M=8)
    with pytest.raises(ValueError):
        _lib.fmm_matvec_host(t, _lib.IMQ, 2.0, np.zeros((2, 50)), np.zeros((1, 50)), M=8)
    with pytest.raises(ValueError):
        _lib.interp_solve(t, _lib.IMQ, 2.0, f64(50), f64(51))
    with pytest.raises(ValueError):
        _lib.interp_solve(t, _lib.IMQ, 2.0, f64(2, 50), f64(50))
    with pytest.raises(TypeError):
        _lib.interp_solve(t, _lib.IMQ, 2.0, f64(2, 50), f64(2, 50))


def test_direct_sum_and_ordering_shapes():
    X = f64(40, 3)
    tg = torch.zeros(5, dtype=torch.int64)
    with pytest.raises(TypeError):
        _lib.direct_sum(X, _lib.IMQ, 2.0, f64(40), tg, f64(5))
    with pytest.raises(ValueError):
        _lib.direct_sum(X, _lib.IMQ, 2.0, f64(39), tg, f64(5))
    with pytest.raises(ValueError):
        _lib.direct_sum(X, _lib.IMQ, 2.0, f64(40), tg, f64(4))
    with pytest.raises(ValueError):
        _lib.direct_sum(f64(120), _lib.IMQ, 2.0, f64(40), tg, f64(5))
    perm = torch.zeros(40, dtype=torch.int32)
    keys = torch.zeros(40, dtype=torch.int64)
    with pytest.raises(ValueError):
        _lib.morton_order_noalloc(X, np.zeros(3), 1.0, 3, perm[:39], keys)
    with pytest.raises(ValueError):
        _lib.morton_order_noalloc(X, np.zeros(3), 1.0, 3, perm, keys[:39])


def test_preconditioner_and_network_shapes():
    t = FakeTree(64, 2)
    with pytest.raises(ValueError):
        _lib.precond_apply(t, f64(64), f64(63))
    with pytest.raises(ValueError):
        _lib.precond_features(t, 2.0, np.arange(5), torch.zeros((5, 32 * 3), dtype=torch.float32))
    net = _lib.Mlp.__new__(_lib.Mlp)          # shape logic only: no handle, no library call
    net._h = None
    net.d_in, net.width, net.d_out = 64, 128, 32
    X = torch.zeros((10, 64), dtype=torch.float32)
    with pytest.raises(ValueError):
        net.forward(torch.zeros((10, 63), dtype=torch.float32), torch.zeros((10, 32)))
    with pytest.raises(ValueError):
        net.forward(X, torch.zeros((9, 32), dtype=torch.float32))
    with pytest.raises(ValueError):
        net.train_step(X, torch.zeros((10, 31), dtype=torch.float32), 1e-3)
    with pytest.raises(TypeError):
        net.forward(X, torch.zeros((10, 32), dtype=torch.float32))


def test_parameter_block():
    """No explicit parameter: NULL (the library's defaults).  Any explicit one,
    including csample=0 alone, gives a full block with the same defaults filled in."""
    assert _lib._params() is None
    p = _lib._params(csample=0, kernel=_lib.GAUSSIAN, side=2.0)
    assert p is not None and p.csample == 0
    assert (p.M, p.period_L, p.window_alpha, p.grid) == (32, 8.0, 0.0, _lib.GRID_SHARED)
    q = _lib._params(M=16, kernel=_lib.IMQ)
    assert (q.M, q.period_L, q.window_alpha, q.csample) == (16, 4.0, 4.5, 1)
    n = _lib._params(grid=_lib.GRID_NESTED, lagrange_K=6, kernel=_lib.MQ)
    assert (n.grid, n.lagrange_K, n.window_alpha) == (_lib.GRID_NESTED, 6, 4.5)
