"""Thin ctypes binding of libh2ulv.so (argument marshalling only).

The functions carry the C ABI's names and arguments (include/h2ulv.h).
Arrays may be torch tensors (host or CUDA; their data pointers are passed)
or numpy arrays (host).  Every computation runs in the CUDA library; if the
library is missing this module raises instead of falling back to anything.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libh2ulv.so")

H2_OK, H2_ERR_ARG, H2_ERR_NONFINITE, H2_ERR_OOM, H2_ERR_BUDGET = 0, 1, 2, 3, 4
H2_ERR_SINGULAR, H2_ERR_RANK_CAP, H2_ERR_NOT_CONVERGED, H2_ERR_DEVICE = 5, 6, 7, 8
H2_ERR_STATE, H2_ERR_NOT_SPD, H2_ERR_TIMEOUT = 9, 10, 11
H2_K_LAPLACE, H2_K_YUKAWA, H2_K_MATERN32 = 0, 1, 2
H2_FP64, H2_MIXED = 0, 1
KERNEL_KIND = {"laplace": H2_K_LAPLACE, "yukawa": H2_K_YUKAWA, "matern32": H2_K_MATERN32}

EXPORTED = ("h2_construct", "h2_construct_batched", "h2_factor", "h2_solve", "h2_solve_batched", "h2_matvec",
            "h2_logdet", "h2_logdet_noalloc", "h2_stats", "h2_profile", "h2_last_error", "h2_destroy",
            "h2_mlp_param_count", "h2_mlp_create", "h2_mlp_train", "h2_mlp_forward", "h2_mlp_gradient",
            "h2_mlp_params", "h2_mlp_last_error", "h2_mlp_destroy", "h2_box_features", "h2_set_rank_predictor")


class h2_kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("delta", ctypes.c_double), ("kappa", ctypes.c_double),
                ("ell", ctypes.c_double), ("nugget", ctypes.c_double)]


class h2_options(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("leaf", ctypes.c_int32), ("tol", ctypes.c_double),
                ("max_rank", ctypes.c_int32), ("far_s0", ctypes.c_int32), ("far_smin", ctypes.c_int32),
                ("hbm_budget_bytes", ctypes.c_int64), ("partition", ctypes.c_int32)]


class H2Error(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"h2 status {status}: {msg}")
        self.status = status


_lib = None


def lib():
    """Load libh2ulv.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.h2_construct.argtypes = [vp, i64, ctypes.POINTER(h2_kernel), ctypes.POINTER(h2_options), vp,
                                   ctypes.POINTER(vp)]
        L.h2_construct_batched.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(i64), ctypes.POINTER(h2_kernel),
                                           ctypes.POINTER(h2_options), vp, ctypes.POINTER(vp)]
        L.h2_factor.argtypes = [vp, i32, i32]
        L.h2_solve.argtypes = [vp, vp, vp, i32, i64, dp, i32, vp, ctypes.POINTER(i32)]
        L.h2_solve_batched.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32),
                                       ctypes.POINTER(i64), dp, i32, vp, ctypes.POINTER(i32)]
        L.h2_matvec.argtypes = [vp, vp, vp, i32, i64]
        L.h2_logdet.argtypes = [vp, vp, vp]
        L.h2_logdet_noalloc.argtypes = [vp, vp, vp]
        L.h2_stats.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
        L.h2_profile.argtypes = [i32, i32]
        fp = ctypes.c_float
        L.h2_mlp_param_count.argtypes = [i32]
        L.h2_mlp_param_count.restype = i32
        L.h2_mlp_create.argtypes = [i32, vp, vp, ctypes.POINTER(vp)]
        L.h2_mlp_train.argtypes = [vp, vp, vp, i32, i32, fp, vp]
        L.h2_mlp_forward.argtypes = [vp, vp, i32, vp]
        L.h2_mlp_gradient.argtypes = [vp, vp, vp, i32, vp, vp]
        L.h2_mlp_params.argtypes = [vp, vp]
        L.h2_mlp_last_error.restype = ctypes.c_char_p
        L.h2_mlp_destroy.argtypes = [vp]
        L.h2_box_features.argtypes = [vp, i32, vp, vp, ctypes.POINTER(i32)]
        L.h2_set_rank_predictor.argtypes = [vp, vp, dp]
        for f in ("h2_mlp_create", "h2_mlp_train", "h2_mlp_forward", "h2_mlp_gradient", "h2_mlp_params",
                  "h2_box_features", "h2_set_rank_predictor"):
            getattr(L, f).restype = ctypes.c_int
        L.h2_last_error.restype = ctypes.c_char_p
        L.h2_destroy.argtypes = [vp]
        for f in ("h2_construct", "h2_construct_batched", "h2_factor", "h2_solve", "h2_solve_batched", "h2_matvec",
                  "h2_logdet",
                  "h2_logdet_noalloc", "h2_stats", "h2_profile"):
            getattr(L, f).restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    """Raw data pointer of a torch tensor or numpy array (must be contiguous)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(type(a))


def _check(st):
    if st != H2_OK:
        raise H2Error(st, lib().h2_last_error().decode())


def make_kernel(kind="laplace", delta=1e-3, kappa=1.0, ell=0.1, nugget=1e-4):
    return h2_kernel(KERNEL_KIND.get(kind, kind), delta, kappa, ell, nugget)


PARTITION = {"bisection": 0, "kmeans": 1}


def make_options(eta=1.0, leaf=256, tol=1e-8, max_rank=128, far_s0=32, far_smin=4, hbm_budget_bytes=0,
                 partition="bisection"):
    return h2_options(eta, leaf, tol, max_rank, far_s0, far_smin, hbm_budget_bytes, PARTITION.get(partition, partition))


def h2_construct(points, N, kernel, options, stream=None):
    """points: N x 3 row-major float64 (host or device).  Returns a handle."""
    h = ctypes.c_void_p()
    _check(lib().h2_construct(_ptr(points), int(N), ctypes.byref(kernel), ctypes.byref(options),
                              ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def h2_construct_batched(points_list, kernel, options, stream=None):
    P = len(points_list)
    ptrs = (ctypes.c_void_p * P)(*[_ptr(p).value for p in points_list])
    Ns = (ctypes.c_int64 * P)(*[int(p.shape[0]) for p in points_list])
    h = ctypes.c_void_p()
    _check(lib().h2_construct_batched(P, ptrs, Ns, ctypes.byref(kernel), ctypes.byref(options),
                                      ctypes.c_void_p(stream or 0), ctypes.byref(h)))
    return h


def h2_factor(h, precision=H2_FP64, spd=0):
    _check(lib().h2_factor(h, int(precision), int(spd)))


def h2_solve(h, b, x, nrhs, ld, target=1e-10, max_iter=20, check=True):
    """Returns (status, achieved relative residuals, corrections applied)."""
    ach = np.zeros(nrhs, dtype=np.float64)
    it = ctypes.c_int32(0)
    st = lib().h2_solve(h, _ptr(b), _ptr(x), int(nrhs), int(ld), float(target), int(max_iter),
                        ctypes.c_void_p(ach.ctypes.data), ctypes.byref(it))
    if check and st not in (H2_OK, H2_ERR_NOT_CONVERGED):
        _check(st)
    return st, ach, it.value


def h2_solve_batched(h, bs, xs, nrhs, lds, target=1e-10, max_iter=20, check=True):
    """Per-problem right-hand sides of a batched handle.  Returns (status,
    per-problem achieved relative residuals, corrections applied)."""
    P = len(bs)
    bp = (ctypes.c_void_p * P)(*[_ptr(b).value for b in bs])
    xp = (ctypes.c_void_p * P)(*[_ptr(x).value for x in xs])
    nr = (ctypes.c_int32 * P)(*[int(v) for v in nrhs])
    ld = (ctypes.c_int64 * P)(*[int(v) for v in lds])
    ach = np.zeros(P, dtype=np.float64)
    it = ctypes.c_int32(0)
    st = lib().h2_solve_batched(h, bp, xp, nr, ld, float(target), int(max_iter), ctypes.c_void_p(ach.ctypes.data),
                                ctypes.byref(it))
    if check and st not in (H2_OK, H2_ERR_NOT_CONVERGED):
        _check(st)
    return st, ach, it.value


def h2_matvec(h, x, y, nrhs, ld):
    _check(lib().h2_matvec(h, _ptr(x), _ptr(y), int(nrhs), int(ld)))


def h2_logdet(h, nproblems=1):
    ld = np.zeros(nproblems, dtype=np.float64)
    sg = np.zeros(nproblems, dtype=np.int32)
    _check(lib().h2_logdet(h, ctypes.c_void_p(ld.ctypes.data), ctypes.c_void_p(sg.ctypes.data)))
    return ld, sg


def h2_logdet_noalloc(h, nproblems=1):
    """Same result as h2_logdet; the library allocates no device memory for it."""
    ld = np.zeros(nproblems, dtype=np.float64)
    sg = np.zeros(nproblems, dtype=np.int32)
    _check(lib().h2_logdet_noalloc(h, ctypes.c_void_p(ld.ctypes.data), ctypes.c_void_p(sg.ctypes.data)))
    return ld, sg


def h2_stats(h, cap=1 << 16):
    buf = ctypes.create_string_buffer(cap)
    _check(lib().h2_stats(h, buf, cap))
    return buf.value.decode()


def h2_profile(enable, reset=0):
    _check(lib().h2_profile(int(enable), int(reset)))


def _check_mlp(st):
    if st != H2_OK:
        raise H2Error(st, lib().h2_mlp_last_error().decode())


def h2_mlp_param_count(n_features=8):
    return lib().h2_mlp_param_count(n_features)


def h2_mlp_create(init_params, stream=None):
    p = np.ascontiguousarray(init_params, dtype=np.float32)
    m = ctypes.c_void_p()
    _check_mlp(lib().h2_mlp_create(8, ctypes.c_void_p(p.ctypes.data), ctypes.c_void_p(stream or 0), ctypes.byref(m)))
    return m


def h2_mlp_train(m, X, T, steps, lr=1e-3):
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    loss = ctypes.c_float(0)
    _check_mlp(lib().h2_mlp_train(m, ctypes.c_void_p(X.ctypes.data), ctypes.c_void_p(T.ctypes.data), len(T),
                                  int(steps), float(lr), ctypes.byref(loss)))
    return loss.value


def h2_mlp_forward(m, X):
    X = np.ascontiguousarray(X, dtype=np.float32)
    Y = np.zeros(len(X), dtype=np.float32)
    _check_mlp(lib().h2_mlp_forward(m, ctypes.c_void_p(X.ctypes.data), len(X), ctypes.c_void_p(Y.ctypes.data)))
    return Y


def h2_mlp_gradient(m, X, T):
    X = np.ascontiguousarray(X, dtype=np.float32)
    T = np.ascontiguousarray(T, dtype=np.float32)
    g = np.zeros(h2_mlp_param_count(), dtype=np.float32)
    loss = ctypes.c_float(0)
    _check_mlp(lib().h2_mlp_gradient(m, ctypes.c_void_p(X.ctypes.data), ctypes.c_void_p(T.ctypes.data), len(T),
                                     ctypes.c_void_p(g.ctypes.data), ctypes.byref(loss)))
    return g, loss.value


def h2_mlp_params(m):
    p = np.zeros(h2_mlp_param_count(), dtype=np.float32)
    _check_mlp(lib().h2_mlp_params(m, ctypes.c_void_p(p.ctypes.data)))
    return p


def h2_mlp_destroy(m):
    lib().h2_mlp_destroy(m)


def h2_box_features(h, height, with_ranks=False):
    nb = ctypes.c_int32(0)
    _check(lib().h2_box_features(h, int(height), None, None, ctypes.byref(nb)))
    F = np.zeros((nb.value, 8), dtype=np.float32)
    R = np.zeros(nb.value, dtype=np.int32) if with_ranks else None
    _check(lib().h2_box_features(h, int(height), ctypes.c_void_p(F.ctypes.data),
                                 ctypes.c_void_p(R.ctypes.data) if with_ranks else None, ctypes.byref(nb)))
    return (F, R) if with_ranks else F


def h2_set_rank_predictor(h, m, margin=0.15):
    _check(lib().h2_set_rank_predictor(h, m, float(margin)))


def h2_destroy(h):
    lib().h2_destroy(h)
