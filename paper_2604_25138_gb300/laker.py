"""Thin Python binding of liblaker's C ABI (include/laker.h).

Argument marshalling only: every computation runs in the CUDA library.  Device
arrays are passed as torch CUDA tensors (float64, contiguous); torch is used
for device memory and the current stream, nothing else.  If the shared library
is missing this module raises on import of the library -- there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblaker.so")

FP64, FP32, BF16X3 = 0, 1, 2
AUTO, MATERIALISED, MATRIX_FREE = 0, 1, 2

OK = 0
ERR_ARG, ERR_CUDA, ERR_NOT_SPD, ERR_BREAKDOWN, ERR_MAXITER = -1, -2, -3, -4, -5
ERR_NONFINITE, ERR_TIMEOUT, ERR_OOM, ERR_UNSUPPORTED = -6, -7, -8, -9


class LakerError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"laker status {status}: {msg}")
        self.status = status


class FitInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("c", ctypes.c_double),
                ("rho", ctypes.c_double), ("change", ctypes.c_double), ("status", ctypes.c_int),
                ("eig_sweeps", ctypes.c_int)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("true_residuals", ctypes.c_int), ("converged", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("rel_res_true", ctypes.c_double), ("status", ctypes.c_int),
                ("restarts", ctypes.c_int)]


class BatchItem(ctypes.Structure):
    _fields_ = [("op", ctypes.c_void_p), ("P", ctypes.c_void_p), ("y", ctypes.c_void_p), ("alpha", ctypes.c_void_p)]


_lib = None


def library() -> ctypes.CDLL:
    """Load liblaker.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"liblaker.so not built ({LIB_PATH}); run paper_2604_25138_gb300/build.py")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, i32, f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    pvp = ctypes.POINTER(ctypes.c_void_p)
    pi32 = ctypes.POINTER(ctypes.c_int)
    sig = {
        "laker_create": (i32, [pvp, i32, vp]),
        "laker_destroy": (i32, [vp]),
        "laker_last_error": (ctypes.c_char_p, [vp]),
        "laker_status_string": (ctypes.c_char_p, [i32]),
        "laker_launch_count": (i64, [vp]),
        "laker_build_kernel": (i32, [vp, vp, i64, i32, f64, f64, i32, i32, pvp]),
        "laker_op_destroy": (i32, [vp]),
        "laker_op_describe": (i32, [vp, pi32, pi32, ctypes.POINTER(f64), ctypes.POINTER(f64)]),
        "laker_pcg_solve_batched": (i32, [vp, i32, ctypes.POINTER(BatchItem), f64, i32, i32,
                                          ctypes.POINTER(SolveInfo), ctypes.POINTER(f64)]),
        "laker_setnet_create": (i32, [vp, i32, i32, i32, ctypes.c_uint64, pvp]),
        "laker_setnet_destroy": (i32, [vp]),
        "laker_setnet_num_params": (i64, [vp]),
        "laker_setnet_get_params": (i32, [vp, vp, vp]),
        "laker_setnet_set_params": (i32, [vp, vp, vp]),
        "laker_setnet_point_features": (i32, [vp, i64, i32, vp, vp, vp, vp]),
        "laker_setnet_forward": (i32, [vp, vp, i32, vp, pi32, vp, pi32, vp, vp]),
        "laker_setnet_gradient": (i32, [vp, vp, i32, vp, pi32, vp, pi32, vp, vp, vp, ctypes.POINTER(ctypes.c_float)]),
        "laker_setnet_train_step": (i32, [vp, vp, i32, vp, pi32, vp, pi32, vp, vp, ctypes.c_float,
                                          ctypes.POINTER(ctypes.c_float)]),
        "laker_precond_direction_features": (i32, [vp, vp, vp]),
        "laker_fit_preconditioner_learned": (i32, [vp, vp, vp, i32, f64, f64, f64, i32, f64, vp, vp, i32, pvp,
                                                   ctypes.POINTER(FitInfo)]),
        "laker_op_matvec": (i32, [vp, vp, vp, vp]),
        "laker_op_matvec_fp64": (i32, [vp, vp, vp, vp]),
        "laker_op_time_operator": (i32, [vp, vp, vp, i32, ctypes.POINTER(f64)]),
        "laker_op_time_product": (i32, [vp, vp, vp, i32, ctypes.POINTER(f64)]),
        "laker_fit_preconditioner": (i32, [vp, vp, vp, i32, f64, f64, f64, i32, f64, pvp,
                                           ctypes.POINTER(FitInfo)]),
        "laker_precond_jacobi": (i32, [vp, vp, pvp]),
        "laker_precond_destroy": (i32, [vp]),
        "laker_precond_apply": (i32, [vp, vp, vp, vp]),
        "laker_precond_export": (i32, [vp, vp, vp, vp, vp]),
        "laker_pcg_solve": (i32, [vp, vp, vp, vp, vp, f64, i32, i32, ctypes.POINTER(SolveInfo)]),
        "laker_pcg_solve_trace": (i32, [vp, vp, vp, vp, vp, f64, i32, i32, ctypes.POINTER(SolveInfo),
                                        ctypes.POINTER(f64), i32]),
        "laker_lanczos_extremes": (i32, [ctypes.POINTER(f64), i32, ctypes.POINTER(f64), ctypes.POINTER(f64)]),
        "laker_trace_gap_iterations": (i32, [ctypes.POINTER(f64), i32, f64, f64]),
        "laker_eval_map": (i32, [vp, vp, vp, i64, vp, vp]),
        "laker_eval_map_method": (i32, [vp, vp, vp, i64, vp, vp, i32]),
        "laker_eval_map_noalloc": (i32, [vp, vp, vp, i64, vp, vp]),
        "laker_fit_preconditioner_seeded": (i32, [vp, vp, ctypes.c_uint64, i32, f64, f64, f64, i32, f64, pvp,
                                                  ctypes.POINTER(FitInfo)]),
        "laker_random_directions": (i32, [vp, ctypes.c_uint64, i64, i32, vp]),
        "laker_philox4x32_10": (i32, [vp, ctypes.c_uint64, ctypes.c_uint64, i64, vp]),
        "laker_pcg_solve_gap": (i32, [vp, vp, vp, vp, vp, f64, f64, f64, i32, i32, ctypes.POINTER(SolveInfo)]),
        "laker_set_wait_budget": (i32, [vp, i64]),
        "laker_gd_solve": (i32, [vp, vp, vp, vp, f64, f64, i32, ctypes.POINTER(f64), ctypes.POINTER(SolveInfo),
                                 ctypes.POINTER(f64), i32]),
        "laker_op_lambda_max": (i32, [vp, vp, i32, ctypes.POINTER(f64)]),
        "laker_prediction_discrepancy": (i32, [vp, vp, vp, vp, ctypes.POINTER(f64)]),
        "laker_setnet_save": (i32, [vp, vp, ctypes.c_char_p]),
        "laker_setnet_load": (i32, [vp, ctypes.c_char_p, pvp]),
        "laker_op_append": (i32, [vp, vp, vp, i64, pvp]),
        "laker_pcg_solve_concurrent": (i32, [vp, i32, ctypes.POINTER(BatchItem), f64, i32, i32, i32,
                                             ctypes.POINTER(SolveInfo), ctypes.POINTER(f64)]),
        "laker_pcg_solve_warm": (i32, [vp, vp, vp, vp, vp, f64, i32, i32, ctypes.POINTER(SolveInfo)]),
        "laker_fit_preconditioner_warm": (i32, [vp, vp, vp, i32, f64, f64, f64, i32, f64, vp, pvp,
                                                ctypes.POINTER(FitInfo)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t: torch.Tensor | None, name: str, numel: int | None = None) -> int | None:
    if t is None:
        return None
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return t.data_ptr()


class Context:
    """laker_create / laker_destroy; binds a device and the current torch stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        lib = library()
        self.device = device
        # The library captures PCG iterations into CUDA graphs, which needs a
        # non-legacy stream; every call below orders this stream after the
        # caller's current stream and the caller's stream after it.
        with torch.cuda.device(device):
            s = stream if stream is not None else torch.cuda.Stream(device)
        self.stream = s
        h = ctypes.c_void_p()
        st = lib.laker_create(ctypes.byref(h), device, ctypes.c_void_p(s.cuda_stream))
        if st != OK:
            raise LakerError(st, "laker_create failed")
        self.handle = h

    def __enter__(self):
        self.stream.wait_stream(torch.cuda.current_stream(self.device))
        return self

    def __exit__(self, *exc):
        torch.cuda.current_stream(self.device).wait_stream(self.stream)
        return False

    def check(self, st: int, allowed=(OK,)):
        if st not in allowed:
            raise LakerError(st, library().laker_last_error(self.handle).decode())
        return st

    def launches(self) -> int:
        return library().laker_launch_count(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            library().laker_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class Operator:
    ctx: Context
    handle: ctypes.c_void_p
    n: int
    d: int
    precision: int
    variant: int
    Q: torch.Tensor

    def close(self):
        if self.handle:
            library().laker_op_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclasses.dataclass
class Preconditioner:
    ctx: Context
    handle: ctypes.c_void_p
    n: int
    n_r: int
    info: dict

    def close(self):
        if self.handle:
            library().laker_precond_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def laker_build_kernel(ctx: Context, Q: torch.Tensor, scale: float, lam: float, precision: int = FP64,
                       variant: int = AUTO) -> Operator:
    n, d = Q.shape
    h = ctypes.c_void_p()
    with ctx:
        ctx.check(library().laker_build_kernel(ctx.handle, _ptr(Q, "Q"), n, d, scale, lam, precision, variant,
                                               ctypes.byref(h)))
    return Operator(ctx, h, n, d, precision, variant, Q)


def laker_op_append(ctx: Context, op: Operator, Q_new: torch.Tensor) -> Operator:
    """Streaming update: the operator over op's points followed by the rows of
    Q_new (m x d), reusing op's stored entries.  op stays valid."""
    m, d = Q_new.shape
    if d != op.d:
        raise ValueError("Q_new has %d columns, the operator %d" % (d, op.d))
    h = ctypes.c_void_p()
    with ctx:
        ctx.check(library().laker_op_append(ctx.handle, op.handle, _ptr(Q_new, "Q_new", m * d), m, ctypes.byref(h)))
    return Operator(ctx, h, op.n + m, d, op.precision, op.variant, torch.cat([op.Q, Q_new]))


def laker_op_describe(op: Operator) -> dict:
    """The operator's precision, the variant its products use and, for an
    FP32 operator built with AUTO, the measured time of each variant (ms)."""
    p, v = ctypes.c_int(), ctypes.c_int()
    tm, tf = ctypes.c_double(), ctypes.c_double()
    st = library().laker_op_describe(op.handle, ctypes.byref(p), ctypes.byref(v), ctypes.byref(tm), ctypes.byref(tf))
    if st != OK:
        raise LakerError(st, "laker_op_describe")
    return {"precision": p.value, "variant": v.value, "t_materialised_ms": tm.value, "t_matrix_free_ms": tf.value}


def laker_op_matvec(ctx: Context, op: Operator, x: torch.Tensor, w: torch.Tensor | None = None,
                    fp64: bool = False) -> torch.Tensor:
    if w is None:
        w = torch.empty_like(x)
    fn = library().laker_op_matvec_fp64 if fp64 else library().laker_op_matvec
    with ctx:
        ctx.check(fn(ctx.handle, op.handle, _ptr(x, "x", op.n), _ptr(w, "w", op.n)))
    return w


def laker_op_time_operator(ctx: Context, op: Operator, x: torch.Tensor, reps: int = 20) -> float:
    """Average device milliseconds of the operator's main kernel (roofline use)."""
    ms = ctypes.c_double()
    with ctx:
        ctx.check(library().laker_op_time_operator(ctx.handle, op.handle, _ptr(x, "x", op.n), reps,
                                                   ctypes.byref(ms)))
    return ms.value


def laker_op_time_product(ctx: Context, op: Operator, x: torch.Tensor, reps: int = 20) -> float:
    """Average device milliseconds of one whole product as PCG issues it."""
    ms = ctypes.c_double()
    with ctx:
        ctx.check(library().laker_op_time_product(ctx.handle, op.handle, _ptr(x, "x", op.n), reps,
                                                  ctypes.byref(ms)))
    return ms.value


def laker_fit_preconditioner(ctx: Context, op: Operator, Z: torch.Tensor, gamma: float = 0.1,
                             rho: float = -1.0, eps: float = 1e-8, max_iter: int = 200,
                             tol: float = 1e-10) -> Preconditioner:
    n, n_r = Z.shape
    info = FitInfo()
    h = ctypes.c_void_p()
    with ctx:
        ctx.check(library().laker_fit_preconditioner(ctx.handle, op.handle, _ptr(Z, "Z", op.n * n_r), n_r, gamma,
                                                     rho, eps, max_iter, tol, ctypes.byref(h), ctypes.byref(info)))
    d = {f: getattr(info, f) for f, _ in FitInfo._fields_}
    return Preconditioner(ctx, h, n, n_r, d)


class SetNet:
    """Handle of the learned set-to-parameters network (device weights)."""

    def __init__(self, ctx: Context, in_dim: int, hidden: int = 256, dir_hidden: int = 64, seed: int = 0,
                 _handle=None):
        self.ctx = ctx
        self.in_dim, self.hidden, self.dir_hidden = in_dim, hidden, dir_hidden
        if _handle is not None:
            self.handle = _handle
            return
        h = ctypes.c_void_p()
        with ctx:
            ctx.check(library().laker_setnet_create(ctx.handle, in_dim, hidden, dir_hidden, seed, ctypes.byref(h)))
        self.handle = h

    def save(self, path: str):
        """laker_setnet_save: weights, Adam moments and step to a file."""
        with self.ctx:
            self.ctx.check(library().laker_setnet_save(self.ctx.handle, self.handle, os.fsencode(path)))

    @staticmethod
    def load(ctx: Context, path: str, in_dim: int, hidden: int = 256, dir_hidden: int = 64) -> "SetNet":
        """laker_setnet_load: a network restored from a checkpoint file (the
        sizes given here must be those stored in it)."""
        h = ctypes.c_void_p()
        with ctx:
            ctx.check(library().laker_setnet_load(ctx.handle, os.fsencode(path), ctypes.byref(h)))
        return SetNet(ctx, in_dim, hidden, dir_hidden, _handle=h)

    def num_params(self) -> int:
        return int(library().laker_setnet_num_params(self.handle))

    def get_params(self):
        import numpy as np
        out = np.empty(self.num_params(), dtype=np.float32)
        with self.ctx:
            self.ctx.check(library().laker_setnet_get_params(self.ctx.handle, self.handle,
                                                             out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def set_params(self, theta):
        import numpy as np
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.size != self.num_params():
            raise ValueError("parameter vector has the wrong size")
        with self.ctx:
            self.ctx.check(library().laker_setnet_set_params(self.ctx.handle, self.handle,
                                                             t.ctypes.data_as(ctypes.c_void_p)))

    def close(self):
        if getattr(self, "handle", None):
            library().laker_setnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _offsets(counts):
    arr = (ctypes.c_int * (len(counts) + 1))()
    s = 0
    arr[0] = 0
    for k, c in enumerate(counts):
        s += int(c)
        arr[k + 1] = s
    return arr


def _f32(t: torch.Tensor, name: str, numel: int | None = None):
    if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements")
    return ctypes.c_void_p(t.data_ptr())


def laker_setnet_point_features(ctx: Context, loc: torch.Tensor, Q: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    n, d = Q.shape
    X = torch.empty((n, d + 3), dtype=torch.float32, device=Q.device)
    with ctx:
        ctx.check(library().laker_setnet_point_features(ctx.handle, n, d, _ptr(loc, "loc", 2 * n), _ptr(Q, "Q"),
                                                        _ptr(y, "y", n), _f32(X, "X")))
    return X


def laker_setnet_forward(ctx: Context, net: SetNet, X: torch.Tensor, n_points, F: torch.Tensor, n_dirs):
    """X: concatenated point features, n_points per instance; F: concatenated
    direction features, n_dirs per instance.  Returns (log c, log D)."""
    B = len(n_points)
    po, ko = _offsets(n_points), _offsets(n_dirs)
    logc = torch.empty(B, dtype=torch.float32, device=X.device)
    logD = torch.empty(max(1, ko[B]), dtype=torch.float32, device=X.device)
    with ctx:
        ctx.check(library().laker_setnet_forward(ctx.handle, net.handle, B, _f32(X, "X"), po, _f32(F, "F"), ko,
                                                 _f32(logc, "logc"), _f32(logD, "logD")))
    return logc, logD[:ko[B]]


def laker_setnet_gradient(ctx: Context, net: SetNet, X, n_points, F, n_dirs, tc: torch.Tensor, tD: torch.Tensor):
    B = len(n_points)
    po, ko = _offsets(n_points), _offsets(n_dirs)
    grad = torch.empty(net.num_params(), dtype=torch.float32, device=X.device)
    loss = ctypes.c_float()
    with ctx:
        ctx.check(library().laker_setnet_gradient(ctx.handle, net.handle, B, _f32(X, "X"), po, _f32(F, "F"), ko,
                                                  _f32(tc, "tc", B), _f32(tD, "tD", ko[B]), _f32(grad, "grad"),
                                                  ctypes.byref(loss)))
    return grad, float(loss.value)


def laker_setnet_train_step(ctx: Context, net: SetNet, X, n_points, F, n_dirs, tc, tD, lr: float) -> float:
    B = len(n_points)
    po, ko = _offsets(n_points), _offsets(n_dirs)
    loss = ctypes.c_float()
    with ctx:
        ctx.check(library().laker_setnet_train_step(ctx.handle, net.handle, B, _f32(X, "X"), po, _f32(F, "F"), ko,
                                                    _f32(tc, "tc", B), _f32(tD, "tD", ko[B]), lr, ctypes.byref(loss)))
    return float(loss.value)


def laker_precond_direction_features(ctx: Context, P: Preconditioner) -> torch.Tensor:
    F = torch.empty((P.n_r, 2), dtype=torch.float32, device="cuda")
    with ctx:
        ctx.check(library().laker_precond_direction_features(ctx.handle, P.handle, _f32(F, "F")))
    return F


def laker_fit_preconditioner_learned(ctx: Context, op: Operator, Z: torch.Tensor, net: SetNet, X: torch.Tensor,
                                     mode: int = 0, gamma: float = 0.1, rho: float = -1.0, eps: float = 1e-8,
                                     max_iter: int = 200, tol: float = 1e-10) -> Preconditioner:
    """mode 0: CCCP iterations started from the network's prediction; mode 1:
    the prediction is used as Sigma_* directly."""
    n, n_r = Z.shape
    info = FitInfo()
    h = ctypes.c_void_p()
    with ctx:
        ctx.check(library().laker_fit_preconditioner_learned(ctx.handle, op.handle, _ptr(Z, "Z", op.n * n_r), n_r,
                                                             gamma, rho, eps, max_iter, tol, net.handle,
                                                             _f32(X, "X", n * net.in_dim), mode, ctypes.byref(h),
                                                             ctypes.byref(info)))
    d = {f: getattr(info, f) for f, _ in FitInfo._fields_}
    return Preconditioner(ctx, h, n, n_r, d)


def laker_precond_jacobi(ctx: Context, op: Operator) -> Preconditioner:
    h = ctypes.c_void_p()
    with ctx:
        ctx.check(library().laker_precond_jacobi(ctx.handle, op.handle, ctypes.byref(h)))
    return Preconditioner(ctx, h, op.n, 0, {})


def laker_precond_apply(ctx: Context, P: Preconditioner, r: torch.Tensor) -> torch.Tensor:
    z = torch.empty_like(r)
    with ctx:
        ctx.check(library().laker_precond_apply(ctx.handle, P.handle, _ptr(r, "r", P.n), _ptr(z, "z", P.n)))
    return z


def laker_precond_export(ctx: Context, P: Preconditioner):
    dev = torch.device("cuda", ctx.device)
    c = torch.empty(1, dtype=torch.float64, device=dev)
    D = torch.empty(P.n_r, dtype=torch.float64, device=dev)
    U = torch.empty(P.n, P.n_r, dtype=torch.float64, device=dev)
    with ctx:
        ctx.check(library().laker_precond_export(ctx.handle, P.handle, c.data_ptr(), D.data_ptr(), U.data_ptr()))
    return float(c.item()), D, U


def laker_pcg_solve(ctx: Context, op: Operator, P: Preconditioner | None, y: torch.Tensor, tol: float,
                    max_iter: int = 100000, refine_every: int = 0, alpha: torch.Tensor | None = None,
                    allow_maxiter: bool = False):
    if alpha is None:
        alpha = torch.empty_like(y)
    info = SolveInfo()
    with ctx:
        st = library().laker_pcg_solve(ctx.handle, op.handle, P.handle if P is not None else None,
                                       _ptr(y, "y", op.n), _ptr(alpha, "alpha", op.n), tol, max_iter, refine_every,
                                       ctypes.byref(info))
    ctx.check(st, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
    return alpha, {f: getattr(info, f) for f, _ in SolveInfo._fields_}


def laker_pcg_solve_trace(ctx: Context, op: Operator, P: Preconditioner | None, y: torch.Tensor, tol: float,
                          max_iter: int = 100000, refine_every: int = 0, alpha: torch.Tensor | None = None,
                          allow_maxiter: bool = False, trace_cap: int | None = None):
    """laker_pcg_solve that also returns the per-product trace as a
    (products x 4) float64 array: delta, |r|^2/|y|^2, R(alpha), beta."""
    import numpy as np
    if alpha is None:
        alpha = torch.empty_like(y)
    cap = int(trace_cap if trace_cap is not None else max_iter)
    trace = np.zeros(4 * cap, dtype=np.float64)
    info = SolveInfo()
    with ctx:
        st = library().laker_pcg_solve_trace(ctx.handle, op.handle, P.handle if P is not None else None,
                                             _ptr(y, "y", op.n), _ptr(alpha, "alpha", op.n), tol, max_iter,
                                             refine_every, ctypes.byref(info),
                                             trace.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cap)
    ctx.check(st, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
    d = {f: getattr(info, f) for f, _ in SolveInfo._fields_}
    rows = min(d["iterations"], cap)
    return alpha, d, trace.reshape(cap, 4)[:rows].copy()


def laker_lanczos_extremes(trace, k: int | None = None):
    """(lmin, lmax) of the Lanczos tridiagonal of the first k rows of a trace."""
    import numpy as np
    t = np.ascontiguousarray(trace, dtype=np.float64)
    k = int(t.shape[0] if k is None else k)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    st = library().laker_lanczos_extremes(t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), k, ctypes.byref(lo),
                                          ctypes.byref(hi))
    if st != OK:
        raise LakerError(st, "laker_lanczos_extremes: bad trace")
    return lo.value, hi.value


def laker_trace_gap_iterations(trace, R_ref: float, gap: float = 1e-3) -> int:
    """First product (1-based) whose objective gap to R_ref is <= gap, or -1."""
    import numpy as np
    t = np.ascontiguousarray(trace, dtype=np.float64)
    return int(library().laker_trace_gap_iterations(t.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), t.shape[0],
                                                    float(R_ref), float(gap)))


def laker_pcg_solve_batched(ctx: Context, items, tol: float, max_iter: int = 100000, refine_every: int = 0,
                            allow_maxiter: bool = False):
    """items: sequence of (op, P or None, y, alpha or None).  Returns the list of
    alphas, the list of info dicts and the per-instance stop times in ms."""
    count = len(items)
    arr = (BatchItem * count)()
    alphas = []
    for k, (op, P, y, alpha) in enumerate(items):
        if alpha is None:
            alpha = torch.empty_like(y)
        alphas.append(alpha)
        arr[k] = BatchItem(op.handle, P.handle if P is not None else None, _ptr(y, "y", op.n),
                           _ptr(alpha, "alpha", op.n))
    infos = (SolveInfo * count)()
    done = (ctypes.c_double * count)()
    with ctx:
        st = library().laker_pcg_solve_batched(ctx.handle, count, arr, tol, max_iter, refine_every, infos, done)
    ctx.check(st, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
    return (alphas, [{f: getattr(infos[k], f) for f, _ in SolveInfo._fields_} for k in range(count)],
            [done[k] for k in range(count)])


def laker_pcg_solve_concurrent(ctx: Context, items, tol: float, max_iter: int = 100000, refine_every: int = 0,
                               streams: int = 16, allow_maxiter: bool = False):
    """items: sequence of (op, P or None, y, alpha or None), solved as concurrent
    single-instance solves on `streams` streams.  Returns the list of alphas,
    the list of info dicts and the per-instance end times in ms (host clock)."""
    count = len(items)
    arr = (BatchItem * count)()
    alphas = []
    for k, (op, P, y, alpha) in enumerate(items):
        if alpha is None:
            alpha = torch.empty_like(y)
        alphas.append(alpha)
        arr[k] = BatchItem(op.handle, P.handle if P is not None else None, _ptr(y, "y", op.n),
                           _ptr(alpha, "alpha", op.n))
    infos = (SolveInfo * count)()
    done = (ctypes.c_double * count)()
    with ctx:
        st = library().laker_pcg_solve_concurrent(ctx.handle, count, arr, tol, max_iter, refine_every, streams,
                                                  infos, done)
    ctx.check(st, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
    return (alphas, [{f: getattr(infos[k], f) for f, _ in SolveInfo._fields_} for k in range(count)],
            [done[k] for k in range(count)])


MAP_AUTO, MAP_DOUBLE_FLOAT, MAP_TENSOR = 0, 1, 2


def laker_eval_map(ctx: Context, op: Operator, Qg: torch.Tensor, alpha: torch.Tensor,
                   out: torch.Tensor | None = None, method: int = MAP_AUTO) -> torch.Tensor:
    m = Qg.shape[0]
    if out is None:
        out = torch.empty(m, dtype=torch.float64, device=alpha.device)
    with ctx:
        ctx.check(library().laker_eval_map_method(ctx.handle, op.handle, _ptr(Qg, "Qg", m * op.d), m,
                                                  _ptr(alpha, "alpha", op.n), _ptr(out, "out", m), int(method)))
    return out


def laker_eval_map_noalloc(ctx: Context, op: Operator, Qg: torch.Tensor, alpha: torch.Tensor,
                           out: torch.Tensor) -> torch.Tensor:
    """Radio map for callers that cannot allocate device memory: the library
    takes its scratch from a static device array (see include/laker.h) and
    `out` must be supplied by the caller."""
    m = Qg.shape[0]
    with ctx:
        ctx.check(library().laker_eval_map_noalloc(ctx.handle, op.handle, _ptr(Qg, "Qg", m * op.d), m,
                                                   _ptr(alpha, "alpha", op.n), _ptr(out, "out", m)))
    return out


def laker_fit_preconditioner_seeded(ctx: Context, op: Operator, seed: int, n_r: int, gamma: float = 0.1,
                                    rho: float = -1.0, eps: float = 1e-8, max_iter: int = 200,
                                    tol: float = 1e-10) -> Preconditioner:
    """CCCP fit with the random directions drawn on the device from `seed`."""
    info = FitInfo()
    h = ctypes.c_void_p()
    with ctx:
        ctx.check(library().laker_fit_preconditioner_seeded(ctx.handle, op.handle, seed, n_r, gamma, rho, eps,
                                                            max_iter, tol, ctypes.byref(h), ctypes.byref(info)))
    d = {f: getattr(info, f) for f, _ in FitInfo._fields_}
    return Preconditioner(ctx, h, op.n, n_r, d)


def laker_fit_preconditioner_warm(ctx: Context, op: Operator, Z: torch.Tensor, prev: Preconditioner,
                                  gamma: float = 0.1, rho: float = -1.0, eps: float = 1e-8, max_iter: int = 200,
                                  tol: float = 1e-10) -> Preconditioner:
    """CCCP fit started from a previous fit's (c, D); Z continues prev's
    directions with rows for the new points."""
    n, n_r = Z.shape
    info = FitInfo()
    h = ctypes.c_void_p()
    with ctx:
        ctx.check(library().laker_fit_preconditioner_warm(ctx.handle, op.handle, _ptr(Z, "Z", op.n * n_r), n_r,
                                                          gamma, rho, eps, max_iter, tol, prev.handle,
                                                          ctypes.byref(h), ctypes.byref(info)))
    d = {f: getattr(info, f) for f, _ in FitInfo._fields_}
    return Preconditioner(ctx, h, op.n, n_r, d)


def laker_pcg_solve_warm(ctx: Context, op: Operator, P: Preconditioner | None, y: torch.Tensor,
                         alpha0: torch.Tensor, tol: float, max_iter: int = 100000, refine_every: int = 0,
                         allow_maxiter: bool = False):
    """PCG from the start alpha0 (not modified); returns (alpha, info)."""
    alpha = alpha0.clone()
    info = SolveInfo()
    with ctx:
        st = library().laker_pcg_solve_warm(ctx.handle, op.handle, P.handle if P is not None else None,
                                            _ptr(y, "y", op.n), _ptr(alpha, "alpha", op.n), tol, max_iter,
                                            refine_every, ctypes.byref(info))
    ctx.check(st, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
    return alpha, {f: getattr(info, f) for f, _ in SolveInfo._fields_}


def laker_random_directions(ctx: Context, seed: int, n: int, n_r: int) -> torch.Tensor:
    Z = torch.empty((n, n_r), dtype=torch.float64, device=torch.device("cuda", ctx.device))
    with ctx:
        ctx.check(library().laker_random_directions(ctx.handle, seed, n, n_r, Z.data_ptr()))
    return Z


def laker_philox4x32_10(ctx: Context, key: int, counter0: int, count: int) -> torch.Tensor:
    """Raw Philox4x32-10 words (count blocks of 4) as an int64 tensor of uint32 values."""
    out = torch.empty(4 * count, dtype=torch.int32, device=torch.device("cuda", ctx.device))
    with ctx:
        ctx.check(library().laker_philox4x32_10(ctx.handle, key, counter0, count, out.data_ptr()))
    return out.to(torch.int64) & 0xFFFFFFFF


def laker_pcg_solve_gap(ctx: Context, op: Operator, P: Preconditioner | None, y: torch.Tensor, R_ref: float,
                        gap: float = 1e-3, tol: float = 0.0, max_iter: int = 100000, refine_every: int = 0,
                        allow_maxiter: bool = False):
    alpha = torch.empty_like(y)
    info = SolveInfo()
    with ctx:
        st = library().laker_pcg_solve_gap(ctx.handle, op.handle, P.handle if P is not None else None,
                                           _ptr(y, "y", op.n), _ptr(alpha, "alpha", op.n), R_ref, gap, tol,
                                           max_iter, refine_every, ctypes.byref(info))
    ctx.check(st, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
    return alpha, {f: getattr(info, f) for f, _ in SolveInfo._fields_}


def laker_set_wait_budget(ctx: Context, cycles: int):
    ctx.check(library().laker_set_wait_budget(ctx.handle, int(cycles)))


def laker_gd_solve(ctx: Context, op: Operator, y: torch.Tensor, eta: float = 0.0, tol: float = 0.0,
                   max_iter: int = 1000, trace_cap: int = 0, allow_maxiter: bool = True):
    """Gradient descent on R(alpha); returns (alpha, info, eta_used, trace)
    with trace a (steps x 2) array of |r|^2/|y|^2 and R(alpha) (or None)."""
    import numpy as np
    alpha = torch.empty_like(y)
    info = SolveInfo()
    eu = ctypes.c_double()
    tr = np.zeros(2 * max(1, trace_cap), dtype=np.float64) if trace_cap > 0 else None
    with ctx:
        st = library().laker_gd_solve(ctx.handle, op.handle, _ptr(y, "y", op.n), _ptr(alpha, "alpha", op.n), eta,
                                      tol, max_iter, ctypes.byref(eu), ctypes.byref(info),
                                      tr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if tr is not None else None,
                                      trace_cap)
    ctx.check(st, (OK, ERR_MAXITER) if allow_maxiter else (OK,))
    d = {f: getattr(info, f) for f, _ in SolveInfo._fields_}
    if tr is not None:
        tr = tr.reshape(trace_cap, 2)[:min(d["iterations"], trace_cap)].copy()
    return alpha, d, eu.value, tr


def laker_op_lambda_max(ctx: Context, op: Operator, iters: int = 50) -> float:
    mu = ctypes.c_double()
    with ctx:
        ctx.check(library().laker_op_lambda_max(ctx.handle, op.handle, iters, ctypes.byref(mu)))
    return mu.value


def laker_prediction_discrepancy(ctx: Context, op: Operator, alpha: torch.Tensor, alpha_ref: torch.Tensor) -> float:
    out = ctypes.c_double()
    with ctx:
        ctx.check(library().laker_prediction_discrepancy(ctx.handle, op.handle, _ptr(alpha, "alpha", op.n),
                                                         _ptr(alpha_ref, "alpha_ref", op.n), ctypes.byref(out)))
    return out.value
