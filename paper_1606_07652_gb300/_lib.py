"""ctypes binding of librbf.so: argument marshalling only.

Every function mirrors an entry point of include/rbf.h.  Device vectors are
torch CUDA tensors (their data_ptr is passed); host vectors are numpy arrays.
Work is enqueued on torch's current CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

GAUSSIAN = 0
IMQ = 1
MQ = 2
WENDLAND = 3
FP64 = 0
FP32 = 1
MAX_DIM = 6
MAX_DEPTH = 10
GRID_SHARED = 0
GRID_NESTED = 1

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "librbf.so")
_lib = None

_c_int, _c_i64, _c_dbl, _c_vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p


class FmmParams(ctypes.Structure):
    _fields_ = [("M", _c_int), ("period_L", _c_dbl), ("window_alpha", _c_dbl), ("csample", _c_int),
                ("grid", _c_int), ("lagrange_K", _c_int)]


class TreeInfo(ctypes.Structure):
    _fields_ = [("N", _c_i64), ("d", _c_int), ("depth", _c_int), ("lo", _c_dbl * MAX_DIM),
                ("side", _c_dbl), ("n_leaf", _c_i64), ("n_near", _c_i64),
                ("max_leaf_points", _c_i64), ("n_box", _c_i64 * (MAX_DEPTH + 1))]


class SolveOpts(ctypes.Structure):
    _fields_ = [("restart_m", _c_int), ("max_iters", _c_int), ("max_refine", _c_int),
                ("rtol", _c_dbl), ("inner_prec", _c_int), ("precond", _c_int),
                ("history_host", ctypes.POINTER(_c_dbl)), ("history_cap", _c_int)]


class SolveReport(ctypes.Structure):
    _fields_ = [("iters", _c_int), ("refinements", _c_int), ("used_fallback", _c_int),
                ("rel_resid", _c_dbl), ("seconds", _c_dbl), ("matvecs_inner", _c_int),
                ("matvecs_fp64", _c_int), ("history_len", _c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("X", _c_vp), ("N", _c_i64), ("d", _c_int), ("kernel", _c_int), ("eps", _c_dbl),
                ("nrhs", _c_int)]


class CostModel(ctypes.Structure):
    _fields_ = [("direct_pair_s", _c_dbl), ("near_pair_s", _c_dbl), ("point_mode_s", _c_dbl),
                ("leaf_mode_s", _c_dbl), ("column_fixed_s", _c_dbl)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class BatchOpts(ctypes.Structure):
    _fields_ = [("tol_kernel", _c_dbl), ("choice", _c_int), ("model", ctypes.POINTER(CostModel))]


class BatchStats(ctypes.Structure):
    _fields_ = [("n_direct", _c_int), ("n_near_only", _c_int), ("n_fmm", _c_int),
                ("direct_items", _c_int), ("product_nodes", _c_int), ("step_nodes", _c_int),
                ("setup_s", _c_dbl), ("predicted_ms", _c_dbl), ("model", CostModel),
                ("direct_pairs", _c_dbl)]


BATCH_AUTO, BATCH_FMM, BATCH_DIRECT = 0, 1, 2


class TrainOpts(ctypes.Structure):
    _fields_ = [("n_train", _c_int), ("epochs", _c_int), ("batch", _c_int), ("lr", ctypes.c_float),
                ("delta_rel", _c_dbl)]


class TrainReport(ctypes.Structure):
    _fields_ = [("loss_first", ctypes.c_float), ("loss_last", ctypes.c_float), ("steps", _c_int),
                ("seconds", _c_dbl)]


class RbfError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = load().rbf_last_error().decode(errors="replace")
        super().__init__(f"{where}: {load().rbf_strerror(code).decode()} ({code}): {msg}")


def library_path() -> str:
    return _LIB_PATH


def load():
    """Load librbf.so (built by __graft_entry__.build() or paper_1606_07652_gb300/build.py)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"librbf.so not built ({_LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.POINTER
    lib.rbf_tree_build.argtypes = [_c_vp, _c_i64, _c_int, _c_vp, _c_dbl, _c_int, _c_vp,
                                   P(_c_vp)]
    lib.rbf_tree_get_info.argtypes = [_c_vp, P(TreeInfo)]
    lib.rbf_tree_export.argtypes = [_c_vp] + [_c_vp] * 6 + [_c_vp]
    lib.rbf_tree_export_level.argtypes = [_c_vp, _c_int, _c_vp, _c_vp, _c_vp, P(_c_i64), _c_vp]
    lib.rbf_fmm_matvec.argtypes = [_c_vp, _c_int, _c_dbl, P(FmmParams), _c_int, _c_vp, _c_i64,
                                   _c_vp, _c_i64, _c_int, _c_vp]
    lib.rbf_check_device_waits.argtypes = []
    lib.rbf_selftest_bounded_wait.argtypes = [_c_dbl, ctypes.POINTER(_c_int), _c_vp]
    lib.rbf_fmm_matvec_host.argtypes = [_c_vp, _c_int, _c_dbl, P(FmmParams), _c_int, _c_vp,
                                        _c_vp, _c_int, _c_vp]
    lib.rbf_direct_sum.argtypes = [_c_vp, _c_i64, _c_int, _c_int, _c_dbl, _c_vp, _c_vp, _c_i64,
                                   _c_vp, _c_vp]
    lib.rbf_interp_solve.argtypes = [_c_vp, _c_int, _c_dbl, P(FmmParams), _c_vp, _c_vp, _c_int,
                                     P(SolveOpts), P(SolveReport), _c_vp]
    lib.rbf_morton_order_noalloc.argtypes = [_c_vp, _c_i64, _c_int, _c_vp, _c_dbl, _c_int, _c_vp,
                                             _c_vp, _c_vp]
    lib.rbf_peak_probe.argtypes = [_c_int, _c_dbl, P(_c_dbl), _c_vp]
    lib.rbf_knn.argtypes = [_c_vp, _c_vp, _c_vp]
    lib.rbf_cardinal_weights.argtypes = [_c_vp, _c_int, _c_dbl, _c_dbl, _c_vp, _c_i64, _c_vp, _c_vp]
    lib.rbf_precond_features.argtypes = [_c_vp, _c_dbl, _c_vp, _c_i64, _c_vp, _c_vp]
    lib.rbf_mlp_create.argtypes = [_c_int, _c_int, _c_int, ctypes.c_uint64, P(_c_vp)]
    lib.rbf_mlp_num_params.argtypes = [_c_vp, P(_c_i64)]
    lib.rbf_mlp_get_params.argtypes = [_c_vp, _c_vp]
    lib.rbf_mlp_set_params.argtypes = [_c_vp, _c_vp]
    lib.rbf_mlp_forward.argtypes = [_c_vp, _c_vp, _c_i64, _c_vp, _c_vp]
    lib.rbf_mlp_gradient.argtypes = [_c_vp, _c_vp, _c_vp, _c_i64, _c_vp, P(ctypes.c_float), _c_vp]
    lib.rbf_mlp_train_step.argtypes = [_c_vp, _c_vp, _c_vp, _c_i64, ctypes.c_float,
                                       P(ctypes.c_float), _c_vp]
    lib.rbf_mlp_save.argtypes = [_c_vp, ctypes.c_char_p]
    lib.rbf_mlp_load.argtypes = [ctypes.c_char_p, P(_c_vp)]
    lib.rbf_mlp_free.argtypes = [_c_vp]
    lib.rbf_mlp_free.restype = None
    lib.rbf_precond_train.argtypes = [_c_vp, _c_int, _c_dbl, _c_vp, P(TrainOpts), P(TrainReport),
                                      _c_vp]
    lib.rbf_precond_build.argtypes = [_c_vp, _c_int, _c_dbl, _c_vp, _c_dbl, _c_vp]
    lib.rbf_precond_apply.argtypes = [_c_vp, _c_vp, _c_vp, _c_vp]
    lib.rbf_eval_create.argtypes = [_c_vp, _c_vp, _c_i64, _c_vp, P(_c_vp)]
    lib.rbf_eval_apply.argtypes = [_c_vp, _c_int, _c_dbl, P(FmmParams), _c_int, _c_vp, _c_i64,
                                   _c_vp, _c_i64, _c_int, _c_vp]
    lib.rbf_eval_free.argtypes = [_c_vp]
    lib.rbf_eval_free.restype = None
    lib.rbf_kernel_error.argtypes = [_c_int, _c_dbl, _c_int, P(FmmParams), _c_dbl, _c_int,
                                     P(_c_dbl)]
    lib.rbf_autotune.argtypes = [_c_int, _c_dbl, _c_int, _c_i64, _c_dbl, _c_dbl, P(FmmParams),
                                 P(_c_int), P(_c_dbl)]
    lib.rbf_batch_create.argtypes = [_c_vp, _c_int, _c_dbl, _c_vp, P(_c_vp)]
    lib.rbf_batch_create_opts.argtypes = [_c_vp, _c_int, P(BatchOpts), _c_vp, P(_c_vp)]
    lib.rbf_batch_get_stats.argtypes = [_c_vp, P(BatchStats)]
    lib.rbf_batch_time_parts.argtypes = [_c_vp, _c_int, _c_int, P(_c_dbl), P(_c_dbl), _c_vp]
    lib.rbf_cost_calibrate.argtypes = [P(CostModel), _c_vp]
    lib.rbf_autotune_cost.argtypes = [_c_int, _c_dbl, _c_int, _c_i64, _c_int, _c_dbl, _c_dbl,
                                      P(CostModel), P(FmmParams), P(_c_int), P(_c_dbl), P(_c_dbl)]
    lib.rbf_batch_layout.argtypes = [_c_vp, _c_vp, _c_vp, _c_vp, P(_c_i64)]
    lib.rbf_batch_matvec.argtypes = [_c_vp, _c_int, _c_vp, _c_vp, _c_vp]
    lib.rbf_batch_solve.argtypes = [_c_vp, _c_vp, _c_vp, _c_int, _c_int, _c_dbl, _c_int, _c_vp,
                                    P(_c_int), P(_c_dbl), _c_vp]
    lib.rbf_batch_free.argtypes = [_c_vp]
    lib.rbf_batch_free.restype = None
    lib.rbf_profile.argtypes = [_c_vp, _c_int]
    lib.rbf_p2m_launch_shape.argtypes = [_c_vp, P(_c_int)]
    lib.rbf_profile_read.argtypes = [_c_vp, _c_vp, _c_vp]
    lib.rbf_tree_free.argtypes = [_c_vp]
    lib.rbf_tree_free.restype = None
    lib.rbf_strerror.argtypes = [_c_int]
    lib.rbf_strerror.restype = ctypes.c_char_p
    lib.rbf_last_error.restype = ctypes.c_char_p
    lib.rbf_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(code, where):
    if code != 0:
        raise RbfError(code, where)


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype_name, where):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{where}: expected a CUDA tensor")
    if str(t.dtype) != f"torch.{dtype_name}":
        raise TypeError(f"{where}: expected {dtype_name}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{where}: tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _rows_cols(a, where):
    """(rows, length) of a (length,) or (rows, length) array or tensor."""
    shape = tuple(a.shape)
    if len(shape) == 1:
        return 1, shape[0]
    if len(shape) == 2:
        return shape[0], shape[1]
    raise ValueError(f"{where}: expected shape (n,) or (nrhs, n), got {shape}")


def _expect(a, shape, where):
    """The library writes and reads whole blocks through raw pointers, so every
    buffer's shape is checked here, before any call."""
    if tuple(a.shape) != tuple(shape):
        raise ValueError(f"{where}: expected shape {tuple(shape)}, got {tuple(a.shape)}")


def _block(tree_n, lam, u, names):
    """nrhs of a (N,) / (nrhs, N) coefficient block and its equally shaped output."""
    nrhs, n = _rows_cols(lam, names[0])
    if n != tree_n:
        raise ValueError(f"{names[0]}: {n} entries per column, the tree has N={tree_n}")
    _expect(u, lam.shape, names[1])
    return nrhs


def version() -> str:
    return load().rbf_version().decode()


def _params(M=None, period_L=None, window_alpha=None, csample=1, kernel=GAUSSIAN, side=1.0,
            grid=GRID_SHARED, lagrange_K=0):
    if (M is None and period_L is None and window_alpha is None and grid == GRID_SHARED
            and int(csample) == 1 and not lagrange_K):
        return None            # the library's defaults
    p = FmmParams()
    p.M = 32 if M is None else int(M)
    p.period_L = 4.0 * side if period_L is None else float(period_L)
    if window_alpha is None:
        window_alpha = 0.0 if kernel == GAUSSIAN else 4.5
    p.window_alpha = float(window_alpha)
    p.csample = int(csample)
    p.grid = int(grid)
    p.lagrange_K = int(lagrange_K)
    return p


class Tree:
    """Owner of an rbf_tree handle (freed with rbf_tree_free)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def info(self) -> dict:
        inf = TreeInfo()
        _check(load().rbf_tree_get_info(self._h, ctypes.byref(inf)), "rbf_tree_get_info")
        d = inf.d
        return {"N": inf.N, "d": d, "depth": inf.depth, "lo": list(inf.lo)[:d], "side": inf.side,
                "n_leaf": inf.n_leaf, "n_near": inf.n_near, "max_leaf_points": inf.max_leaf_points,
                "n_box": list(inf.n_box)[:inf.depth + 1]}

    def export(self) -> dict:
        inf = self.info()
        N, nl, nn = inf["N"], inf["n_leaf"], inf["n_near"]
        out = {"perm": np.empty(N, np.int64), "keys": np.empty(N, np.uint64),
               "leaf_key": np.empty(nl, np.uint64), "leaf_off": np.empty(nl + 1, np.int64),
               "near_off": np.empty(nl + 1, np.int64), "near_idx": np.empty(max(nn, 1), np.int64)}
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
        _check(load().rbf_tree_export(self._h, ptr(out["perm"]), ptr(out["keys"]),
                                      ptr(out["leaf_key"]), ptr(out["leaf_off"]),
                                      ptr(out["near_off"]), ptr(out["near_idx"]), _stream()),
               "rbf_tree_export")
        out["near_idx"] = out["near_idx"][:nn]
        return out

    def export_level(self, level: int) -> dict:
        inf = self.info()
        n_il = _c_i64(0)
        lib = load()
        _check(lib.rbf_tree_export_level(self._h, level, None, None, None, ctypes.byref(n_il),
                                         _stream()), "rbf_tree_export_level")
        nb = inf["n_box"][level]
        key = np.empty(nb, np.uint64)
        off = np.empty(nb + 1, np.int64)
        idx = np.empty(max(n_il.value, 1), np.int64)
        ptr = lambda a: ctypes.c_void_p(a.ctypes.data)
        _check(lib.rbf_tree_export_level(self._h, level, ptr(key), ptr(off), ptr(idx),
                                         ctypes.byref(n_il), _stream()), "rbf_tree_export_level")
        return {"key": key, "il_off": off, "il_idx": idx[:n_il.value]}

    def free(self):
        if self._h:
            load().rbf_tree_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def tree_build(X, lo=None, side=1.0, depth=-1) -> Tree:
    """rbf_tree_build: X is a contiguous float64 CUDA tensor of shape (N, d)."""
    N, d = X.shape
    px = _dev(X, "float64", "tree_build X")
    lo_arr = None
    if lo is not None:
        lo_arr = (ctypes.c_double * d)(*[float(v) for v in np.asarray(lo).reshape(d)])
    h = ctypes.c_void_p()
    _check(load().rbf_tree_build(px, N, d, lo_arr, float(side), int(depth), _stream(),
                                 ctypes.byref(h)), "rbf_tree_build")
    return Tree(h)


def fmm_matvec(tree: Tree, kernel: int, eps: float, lam, u, prec=FP64, M=None, period_L=None,
               window_alpha=None, csample=1, grid=GRID_SHARED, lagrange_K=0):
    """rbf_fmm_matvec: lam, u are float64 CUDA tensors (N,) or (nrhs, N) (rows = columns of
    the column-major N x nrhs block)."""
    info = tree.info()
    N = info["N"]
    nrhs = _block(N, lam, u, ("lam", "u"))
    p = _params(M, period_L, window_alpha, csample, kernel, info["side"], grid, lagrange_K)
    _check(load().rbf_fmm_matvec(tree.handle, kernel, float(eps),
                                 ctypes.byref(p) if p is not None else None, prec,
                                 _dev(lam, "float64", "lam"), N, _dev(u, "float64", "u"), N, nrhs,
                                 _stream()), "rbf_fmm_matvec")
    return u


class Evaluator:
    """rbf_eval handle: the FMM evaluation of a tree's centres at new points Y
    (contiguous float64 CUDA tensor (nt, d) inside the tree's root cube)."""

    def __init__(self, tree: Tree, Y):
        info = tree.info()
        if Y.dim() != 2 or Y.shape[1] != info["d"]:
            raise ValueError(f"Evaluator Y: expected shape (nt, {info['d']}), got {tuple(Y.shape)}")
        nt, d = Y.shape
        h = ctypes.c_void_p()
        _check(load().rbf_eval_create(tree.handle, _dev(Y, "float64", "Evaluator Y"), nt, _stream(),
                                      ctypes.byref(h)), "rbf_eval_create")
        self._h = h
        self.nt = nt
        self.n = info["N"]
        self.side = info["side"]

    def apply(self, kernel: int, eps: float, lam, s, prec=FP64, M=None, period_L=None,
              window_alpha=None, csample=1, grid=GRID_SHARED, lagrange_K=0):
        """rbf_eval_apply: lam float64 CUDA (N,) or (nrhs, N); s float64 CUDA (nt,) or (nrhs, nt)."""
        nrhs, n = _rows_cols(lam, "lam")
        if n != self.n:
            raise ValueError(f"lam: {n} entries per column, the tree has N={self.n}")
        _expect(s, (self.nt,) if lam.dim() == 1 else (nrhs, self.nt), "s")
        p = _params(M, period_L, window_alpha, csample, kernel, self.side, grid, lagrange_K)
        _check(load().rbf_eval_apply(self._h, kernel, float(eps),
                                     ctypes.byref(p) if p is not None else None, prec,
                                     _dev(lam, "float64", "lam"), lam.shape[-1],
                                     _dev(s, "float64", "s"), s.shape[-1], nrhs, _stream()),
               "rbf_eval_apply")
        return s

    def free(self):
        if self._h:
            load().rbf_eval_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def selftest_bounded_wait(seconds: float = 0.05) -> int:
    """rbf_selftest_bounded_wait: 1 when a wait on a barrier that nothing completes gave up."""
    g = _c_int(0)
    _check(load().rbf_selftest_bounded_wait(float(seconds), ctypes.byref(g), _stream()),
           "rbf_selftest_bounded_wait")
    return g.value


def check_device_waits():
    """rbf_check_device_waits: raises when a bounded wait of a tensor-core kernel gave up."""
    _check(load().rbf_check_device_waits(), "rbf_check_device_waits")


def _host_ptr(a, where):
    """Host pointer of a contiguous float64 numpy array or torch CPU tensor (pinned or not)."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{where}: expected a contiguous float64 array")
        return ctypes.c_void_p(a.ctypes.data)
    import torch
    if not isinstance(a, torch.Tensor) or a.is_cuda or a.dtype != torch.float64 \
            or not a.is_contiguous():
        raise TypeError(f"{where}: expected a contiguous float64 host tensor")
    return ctypes.c_void_p(a.data_ptr())


def fmm_matvec_host(tree: Tree, kernel: int, eps: float, lam_host, u_host=None, prec=FP64,
                    M=None, period_L=None, window_alpha=None, csample=1, grid=GRID_SHARED,
                    lagrange_K=0):
    """rbf_fmm_matvec_host: host float64 in (numpy or torch CPU, e.g. pinned), host out;
    the host <-> device copies happen inside the call."""
    if isinstance(lam_host, np.ndarray):
        lam_host = np.ascontiguousarray(lam_host, dtype=np.float64)
    if u_host is None:
        u_host = np.empty(tuple(lam_host.shape), dtype=np.float64)
    info = tree.info()
    nrhs = _block(info["N"], lam_host, u_host, ("lam_host", "u_host"))
    p = _params(M, period_L, window_alpha, csample, kernel, info["side"], grid, lagrange_K)
    _check(load().rbf_fmm_matvec_host(tree.handle, kernel, float(eps),
                                      ctypes.byref(p) if p is not None else None, prec,
                                      _host_ptr(lam_host, "lam_host"), _host_ptr(u_host, "u_host"),
                                      nrhs, _stream()), "rbf_fmm_matvec_host")
    return u_host


def profile(tree: Tree, enable: bool = True):
    """rbf_profile: start (and clear) or stop per-pass event timing."""
    _check(load().rbf_profile(tree.handle, int(bool(enable))), "rbf_profile")


def p2m_launch_shape(tree: Tree) -> int:
    """rbf_p2m_launch_shape: 1 dense, 2 wide (measured), 0 by rule."""
    v = _c_int(0)
    _check(load().rbf_p2m_launch_shape(tree.handle, ctypes.byref(v)), "rbf_p2m_launch_shape")
    return v.value


PASS_NAMES = ("p2p", "p2m", "m2m", "m2l", "l2p", "perm")


def profile_read(tree: Tree) -> dict:
    """rbf_profile_read: per pass {"ms": summed milliseconds, "launches": kernel launches}."""
    ms = (ctypes.c_double * len(PASS_NAMES))()
    nl = (ctypes.c_int64 * len(PASS_NAMES))()
    _check(load().rbf_profile_read(tree.handle, ms, nl), "rbf_profile_read")
    return {n: {"ms": ms[i], "launches": nl[i]} for i, n in enumerate(PASS_NAMES)}


def direct_sum(X, kernel: int, eps: float, lam, targets, u):
    """rbf_direct_sum: X (N, d) float64, lam (N,), targets (nt,) int64, u (nt,) CUDA tensors."""
    if X.dim() != 2:
        raise ValueError(f"X: expected shape (N, d), got {tuple(X.shape)}")
    N, d = X.shape
    _expect(lam, (N,), "lam")
    if targets.dim() != 1:
        raise ValueError(f"targets: expected shape (nt,), got {tuple(targets.shape)}")
    _expect(u, (targets.shape[0],), "u")
    _check(load().rbf_direct_sum(_dev(X, "float64", "X"), N, d, kernel, float(eps),
                                 _dev(lam, "float64", "lam"), _dev(targets, "int64", "targets"),
                                 targets.shape[0], _dev(u, "float64", "u"), _stream()),
           "rbf_direct_sum")
    return u


def interp_solve(tree: Tree, kernel: int, eps: float, u, lam, restart_m=50, max_iters=2000,
                 max_refine=10, rtol=1e-8, inner_prec=FP32, precond=0, M=None, period_L=None,
                 window_alpha=None, csample=1, grid=GRID_SHARED, lagrange_K=0, history=0):
    """rbf_interp_solve: u, lam float64 CUDA tensors (N,) or (nrhs, N); lam holds the guess.
    history > 0 returns up to that many residual-history entries under "history" as
    (iterations, seconds, relative residual, kind) rows, kind 0 = FP64 true residual,
    1 = inner restart residual."""
    info = tree.info()
    nrhs = _block(info["N"], u, lam, ("u", "lam"))
    o = SolveOpts(restart_m, max_iters, max_refine, rtol, inner_prec, precond)
    rep = SolveReport()
    hist = None
    if history > 0:
        hist = (_c_dbl * (4 * int(history)))()
        o.history_host = ctypes.cast(hist, ctypes.POINTER(_c_dbl))
        o.history_cap = int(history)
    p = _params(M, period_L, window_alpha, csample, kernel, info["side"], grid, lagrange_K)
    code = load().rbf_interp_solve(tree.handle, kernel, float(eps),
                                   ctypes.byref(p) if p is not None else None,
                                   _dev(u, "float64", "u"), _dev(lam, "float64", "lam"), nrhs,
                                   ctypes.byref(o), ctypes.byref(rep), _stream())
    report = {"status": code, "iters": rep.iters, "refinements": rep.refinements,
              "used_fallback": rep.used_fallback, "rel_resid": rep.rel_resid,
              "seconds": rep.seconds, "matvecs_inner": rep.matvecs_inner,
              "matvecs_fp64": rep.matvecs_fp64}
    if hist is not None:
        h = np.frombuffer(hist, dtype=np.float64)[:4 * rep.history_len].reshape(-1, 4)
        report["history"] = [[int(r[0]), float(r[1]), float(r[2]), int(r[3])] for r in h]
    if code not in (0, -4):
        raise RbfError(code, "rbf_interp_solve")
    return report


PROBE_FFMA, PROBE_DFMA, PROBE_EX2, PROBE_RSQRT = 0, 1, 2, 3


def peak_probe(kind, seconds=0.3):
    """rbf_peak_probe: measured rate of one arithmetic unit (flop/s for the FMA kinds,
    results/s for the multi-function unit kinds) on the current device."""
    rate = _c_dbl(0.0)
    _check(load().rbf_peak_probe(int(kind), float(seconds), ctypes.byref(rate), _stream()),
           "rbf_peak_probe")
    return rate.value


def morton_order_noalloc(X, lo, side, depth, perm, keys):
    """rbf_morton_order_noalloc: X (N, d) float64, perm (N,) int32 and keys (N,) uint64 or
    int64 CUDA tensors (written).  Allocates no device memory."""
    import torch
    if X.dim() != 2:
        raise ValueError(f"X: expected shape (N, d), got {tuple(X.shape)}")
    N, d = X.shape
    _expect(perm, (N,), "perm")
    _expect(keys, (N,), "keys")
    lo_arr = (ctypes.c_double * d)(*[float(v) for v in np.asarray(lo).reshape(d)])
    if perm.dtype != torch.int32 or keys.dtype not in (torch.int64, torch.uint64):
        raise TypeError("morton_order_noalloc: perm must be int32 and keys 64-bit")
    _check(load().rbf_morton_order_noalloc(_dev(X, "float64", "X"), N, d, lo_arr, float(side),
                                           int(depth), ctypes.c_void_p(perm.data_ptr()),
                                           ctypes.c_void_p(keys.data_ptr()), _stream()),
           "rbf_morton_order_noalloc")


KNN = 32


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def knn(tree: Tree) -> np.ndarray:
    """rbf_knn: (N, 32) int64 original indices of the nearest centres, nearest first."""
    N = tree.info()["N"]
    out = np.empty((N, KNN), dtype=np.int64)
    _check(load().rbf_knn(tree.handle, _np_ptr(out), _stream()), "rbf_knn")
    return out


def cardinal_weights(tree: Tree, kernel: int, eps: float, delta_rel: float, centres) -> np.ndarray:
    """rbf_cardinal_weights: (nc, 32) FP64 local cardinal coefficients."""
    c = np.ascontiguousarray(centres, dtype=np.int64)
    out = np.empty((len(c), KNN), dtype=np.float64)
    _check(load().rbf_cardinal_weights(tree.handle, kernel, float(eps), float(delta_rel), _np_ptr(c),
                                       len(c), _np_ptr(out), _stream()), "rbf_cardinal_weights")
    return out


def precond_features(tree: Tree, eps: float, centres, F):
    """rbf_precond_features into the float32 CUDA tensor F of shape (nc, 32 d)."""
    c = np.ascontiguousarray(centres, dtype=np.int64)
    _expect(F, (len(c), KNN * tree.info()["d"]), "F")
    _check(load().rbf_precond_features(tree.handle, float(eps), _np_ptr(c), len(c),
                                       _dev(F, "float32", "F"), _stream()), "rbf_precond_features")
    return F


class Mlp:
    """Owner of an rbf_mlp handle."""

    def __init__(self, d_in, width, d_out, seed=0):
        h = ctypes.c_void_p()
        _check(load().rbf_mlp_create(d_in, width, d_out, seed, ctypes.byref(h)), "rbf_mlp_create")
        self._h = h
        self.d_in, self.width, self.d_out = d_in, width, d_out

    @property
    def handle(self):
        return self._h

    def num_params(self) -> int:
        n = _c_i64(0)
        _check(load().rbf_mlp_num_params(self._h, ctypes.byref(n)), "rbf_mlp_num_params")
        return n.value

    def get_params(self) -> np.ndarray:
        out = np.empty(self.num_params(), dtype=np.float32)
        _check(load().rbf_mlp_get_params(self._h, _np_ptr(out)), "rbf_mlp_get_params")
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        _expect(p, (self.num_params(),), "params")
        _check(load().rbf_mlp_set_params(self._h, _np_ptr(p)), "rbf_mlp_set_params")

    def _rows(self, X, where="X"):
        if X.dim() != 2 or X.shape[1] != self.d_in:
            raise ValueError(f"{where}: expected shape (n, {self.d_in}), got {tuple(X.shape)}")
        return X.shape[0]

    def forward(self, X, Y):
        _expect(Y, (self._rows(X), self.d_out), "Y")
        _check(load().rbf_mlp_forward(self._h, _dev(X, "float32", "X"), X.shape[0],
                                      _dev(Y, "float32", "Y"), _stream()), "rbf_mlp_forward")
        return Y

    def gradient(self, X, T, G):
        _expect(T, (self._rows(X), self.d_out), "T")
        _expect(G, (self.num_params(),), "G")
        loss = ctypes.c_float(0)
        _check(load().rbf_mlp_gradient(self._h, _dev(X, "float32", "X"), _dev(T, "float32", "T"),
                                       X.shape[0], _dev(G, "float32", "G"), ctypes.byref(loss),
                                       _stream()), "rbf_mlp_gradient")
        return loss.value

    def train_step(self, X, T, lr):
        _expect(T, (self._rows(X), self.d_out), "T")
        loss = ctypes.c_float(0)
        _check(load().rbf_mlp_train_step(self._h, _dev(X, "float32", "X"), _dev(T, "float32", "T"),
                                         X.shape[0], float(lr), ctypes.byref(loss), _stream()),
               "rbf_mlp_train_step")
        return loss.value

    def save(self, path: str):
        """rbf_mlp_save: parameters and Adam state to a checkpoint file."""
        _check(load().rbf_mlp_save(self._h, os.fsencode(path)), "rbf_mlp_save")

    @classmethod
    def load_checkpoint(cls, path: str) -> "Mlp":
        """rbf_mlp_load: a new network from a checkpoint file."""
        h = ctypes.c_void_p()
        _check(load().rbf_mlp_load(os.fsencode(path), ctypes.byref(h)), "rbf_mlp_load")
        net = cls.__new__(cls)
        net._h = h
        n = _c_i64(0)
        _check(load().rbf_mlp_num_params(h, ctypes.byref(n)), "rbf_mlp_num_params")
        with open(path, "rb") as f:
            dims = np.frombuffer(f.read(8 + 20)[8:], dtype=np.int32)
        net.d_in, net.width, net.d_out = int(dims[0]), int(dims[1]), int(dims[4])
        return net

    def free(self):
        if self._h:
            load().rbf_mlp_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def precond_train(tree: Tree, kernel: int, eps: float, net: Mlp, n_train=8192, epochs=200,
                  batch=1024, lr=1e-3, delta_rel=1e-12) -> dict:
    o = TrainOpts(n_train, epochs, batch, lr, delta_rel)
    r = TrainReport()
    _check(load().rbf_precond_train(tree.handle, kernel, float(eps), net.handle, ctypes.byref(o),
                                    ctypes.byref(r), _stream()), "rbf_precond_train")
    return {"loss_first": r.loss_first, "loss_last": r.loss_last, "steps": r.steps,
            "seconds": r.seconds}


def precond_build(tree: Tree, kernel: int, eps: float, net=None, delta_rel=1e-12):
    """rbf_precond_build from the network (net) or exact local solves (net=None)."""
    _check(load().rbf_precond_build(tree.handle, kernel, float(eps),
                                    net.handle if net is not None else None, float(delta_rel),
                                    _stream()), "rbf_precond_build")


def precond_apply(tree: Tree, y, z):
    """rbf_precond_apply: z = P y for float64 CUDA tensors of shape (N,)."""
    N = tree.info()["N"]
    _expect(y, (N,), "y")
    _expect(z, (N,), "z")
    _check(load().rbf_precond_apply(tree.handle, _dev(y, "float64", "y"), _dev(z, "float64", "z"),
                                    _stream()), "rbf_precond_apply")
    return z


def kernel_error(kernel, eps, d, M, period_L, window_alpha, side=1.0, depth=2) -> float:
    """rbf_kernel_error: max |K - Phi| over sampled far offsets."""
    p = FmmParams(M, period_L, window_alpha, 1, GRID_SHARED, 0)
    e = _c_dbl(0)
    _check(load().rbf_kernel_error(kernel, float(eps), d, ctypes.byref(p), float(side), depth,
                                   ctypes.byref(e)), "rbf_kernel_error")
    return e.value


def autotune(kernel, eps, d, N, tol, side=1.0) -> dict:
    p = FmmParams()
    D = _c_int(0)
    e = _c_dbl(0)
    _check(load().rbf_autotune(kernel, float(eps), d, int(N), float(side), float(tol),
                               ctypes.byref(p), ctypes.byref(D), ctypes.byref(e)), "rbf_autotune")
    return {"M": p.M, "period_L": p.period_L, "window_alpha": p.window_alpha, "depth": D.value,
            "err": e.value}


def cost_calibrate() -> CostModel:
    """rbf_cost_calibrate: the FP32 unit costs of this GPU (seconds)."""
    c = CostModel()
    _check(load().rbf_cost_calibrate(ctypes.byref(c), _stream()), "rbf_cost_calibrate")
    return c


def autotune_cost(kernel, eps, d, N, nrhs, tol, model: CostModel, side=1.0) -> dict:
    """rbf_autotune_cost: depth 0 means the direct sum."""
    p = FmmParams()
    D = _c_int(0)
    e = _c_dbl(0)
    t = _c_dbl(0)
    _check(load().rbf_autotune_cost(kernel, float(eps), d, int(N), int(nrhs), float(side),
                                    float(tol), ctypes.byref(model), ctypes.byref(p),
                                    ctypes.byref(D), ctypes.byref(e), ctypes.byref(t)),
           "rbf_autotune_cost")
    return {"M": p.M, "period_L": p.period_L, "window_alpha": p.window_alpha, "depth": D.value,
            "err": e.value, "pred_s": t.value}


class Batch:
    """Owner of an rbf_batch: problems = list of dicts(X=CUDA float64 tensor (N, d), kernel,
    eps, nrhs).  The tensors must outlive the batch.  choice: BATCH_AUTO (cost model),
    BATCH_FMM (a tree and autotuned FMM for every problem) or BATCH_DIRECT."""

    def __init__(self, problems, tol_kernel=1e-6, choice=BATCH_AUTO, model=None):
        arr = (Problem * len(problems))()
        self._keep = []
        for i, q in enumerate(problems):
            X = q["X"]
            self._keep.append(X)
            arr[i] = Problem(_dev(X, "float64", "X"), X.shape[0], X.shape[1], q["kernel"],
                             float(q["eps"]), int(q.get("nrhs", 1)))
        h = ctypes.c_void_p()
        self._model = model
        opts = BatchOpts(float(tol_kernel), int(choice),
                         ctypes.pointer(model) if model is not None else None)
        _check(load().rbf_batch_create_opts(arr, len(problems), ctypes.byref(opts), _stream(),
                                            ctypes.byref(h)), "rbf_batch_create")
        self._h = h
        self.n = len(problems)
        self.problems = problems

    def layout(self):
        off = np.empty(self.n, np.int64)
        dep = np.empty(self.n, np.int32)
        Ms = np.empty(self.n, np.int32)
        tot = _c_i64(0)
        _check(load().rbf_batch_layout(self._h, _np_ptr(off), _np_ptr(dep), _np_ptr(Ms),
                                       ctypes.byref(tot)), "rbf_batch_layout")
        return {"off": off, "depth": dep, "M": Ms, "total": tot.value}

    def stats(self) -> dict:
        st = BatchStats()
        _check(load().rbf_batch_get_stats(self._h, ctypes.byref(st)), "rbf_batch_get_stats")
        out = {k: getattr(st, k) for k, _ in BatchStats._fields_ if k != "model"}
        out["model"] = st.model.as_dict()
        return out

    def time_parts(self, prec=FP32, reps=3) -> dict:
        """rbf_batch_time_parts: device ms of the direct launch and of the tree problems."""
        dm, tm = _c_dbl(0), _c_dbl(0)
        _check(load().rbf_batch_time_parts(self._h, prec, int(reps), ctypes.byref(dm),
                                           ctypes.byref(tm), _stream()), "rbf_batch_time_parts")
        return {"direct_ms": dm.value, "trees_ms": tm.value}

    def _packed(self, *named):
        tot = self.layout()["total"]
        for a, where in named:
            if a.numel() != tot:
                raise ValueError(f"{where}: {a.numel()} entries, the batch packs {tot}")

    def matvec(self, lam, u, prec=FP32):
        """rbf_batch_matvec on packed float64 CUDA tensors of layout()["total"] entries."""
        self._packed((lam, "lam"), (u, "u"))
        _check(load().rbf_batch_matvec(self._h, prec, _dev(lam, "float64", "lam"),
                                       _dev(u, "float64", "u"), _stream()), "rbf_batch_matvec")
        return u

    def solve(self, u, lam, restart_m=30, max_iters=100, rtol=1e-6, prec=FP32):
        self._packed((u, "u"), (lam, "lam"))
        nsys = sum(int(q.get("nrhs", 1)) for q in self.problems)
        rr = np.empty(nsys, np.float64)
        it = _c_int(0)
        ms = _c_dbl(0)
        _check(load().rbf_batch_solve(self._h, _dev(u, "float64", "u"), _dev(lam, "float64", "lam"),
                                      restart_m, max_iters, float(rtol), prec, _np_ptr(rr),
                                      ctypes.byref(it), ctypes.byref(ms), _stream()),
               "rbf_batch_solve")
        return {"rel_resid": rr, "iters": it.value, "step_ms": ms.value}

    def free(self):
        if self._h:
            load().rbf_batch_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
