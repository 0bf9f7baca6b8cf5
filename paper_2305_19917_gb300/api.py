"""Thin ctypes binding of libgbtrsm.so (argument marshalling only).

Functions named ``gb_*`` mirror the C entry points of include/gbtrsm.h one to
one and take raw device pointers (ints) and a stream handle (int, 0 = legacy
default stream).  ``trsm`` / ``trsm_plan`` are conveniences that take torch
CUDA tensors in column-major layout (``stride(0) == 1``) and pass their
pointers and leading dimensions.  Every computation runs in the CUDA
library; there is no CPU path, and loading fails loudly if the library has
not been built.
"""
import ctypes
import os

from . import build as _build

LEFT, RIGHT = 0, 1
LOWER, UPPER = 0, 1
NOTRANS, TRANS = 0, 1
NONUNIT, UNIT = 0, 1
DRIVER_BLOCKED, DRIVER_RECURSIVE, DRIVER_ITERATIVE, DRIVER_AUTO = 0, 1, 2, -1
STATUS_OK, STATUS_NOT_CONVERGED, STATUS_CUDA_ERROR, STATUS_TIMEOUT, STATUS_NO_MODEL = 0, 1, 2, 3, 4
STATUS_SCRATCH_TOO_SMALL = 5
STATUS_RANGE = 6

LIB_PATH = _build.LIB


class GbPlan(ctypes.Structure):
    _fields_ = [("driver", ctypes.c_int32), ("nb", ctypes.c_int32),
                ("depth", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class GbError(RuntimeError):
    def __init__(self, fn, status):
        self.status = status
        super().__init__(f"{fn} returned {status}: {status_string(status)}"
                         + (f" (cuda error {gb_last_cuda_error()})" if status == STATUS_CUDA_ERROR else ""))


_lib = None
i32, i64, dbl, flt, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_float, ctypes.c_void_p

_SIGS = {
    "gb_dtrsm": ([i32, i32, i32, i32, i64, i64, dbl, vp, i64, vp, i64, vp], i32),
    "gb_strsm": ([i32, i32, i32, i32, i64, i64, flt, vp, i64, vp, i64, vp], i32),
    "gb_dtrsm_plan": ([i32, i32, i32, i32, i64, i64, dbl, vp, i64, vp, i64, ctypes.POINTER(GbPlan), vp], i32),
    "gb_strsm_plan": ([i32, i32, i32, i32, i64, i64, flt, vp, i64, vp, i64, ctypes.POINTER(GbPlan), vp], i32),
    "gb_plan_counts": ([ctypes.POINTER(GbPlan), i64, ctypes.POINTER(i64), ctypes.POINTER(i64),
                        ctypes.POINTER(i64), ctypes.POINTER(dbl)], i32),
    "gb_status_string": ([i32], ctypes.c_char_p),
    "gb_last_cuda_error": ([], i32),
    "gb_version": ([], i32),
    "gb_dtrsm_mixed": ([i32, i32, i32, i32, i64, i64, dbl, vp, i64, vp, i64, dbl, i32, i32,
                        ctypes.POINTER(i32), ctypes.POINTER(dbl), vp], i32),
    "gb_dtrsm_mixed_noalloc": ([i32, i32, i32, i32, i64, i64, dbl, vp, i64, vp, i64, dbl, i32, i32,
                                ctypes.POINTER(i32), ctypes.POINTER(dbl), vp], i32),
    "gb_dtrsm_mixed_host": ([i32, i32, i32, i32, i64, i64, dbl, vp, i64, vp, i64, dbl, i32, i32,
                             ctypes.POINTER(i32), ctypes.POINTER(dbl), vp], i32),
    "gb_mixed_host_bytes": ([i32, i32, i64, i64, ctypes.POINTER(i64)], i64),
    "gb_mixed_workspace_release": ([vp], i32),
    "gb_dpotrf": ([i32, i64, vp, i64, ctypes.POINTER(i64), vp], i32),
    "gb_dtrsm_mixed_leaf": ([i32, i32, i32, i32, i64, i64, dbl, vp, i64, vp, i64, dbl, i32, i32, i64,
                             ctypes.POINTER(i32), ctypes.POINTER(dbl), vp], i32),
    "gb_gemm_update": ([i32, i64, i64, i64, vp, i64, vp, i64, vp, i64, dbl, vp], i32),
    "gb_set_lookahead": ([i32], i32),
    "gb_spotrf": ([i32, i64, vp, i64, ctypes.POINTER(i64), vp], i32),
    "gb_trsm_batched": ([i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp], i32),
    "gb_batched_plan_create": ([i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp,
                                ctypes.POINTER(vp)], i32),
    "gb_batched_plan_create_tiled": ([i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp,
                                      ctypes.POINTER(vp)], i32),
    "gb_batched_autotune": ([i32, i64, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp, ctypes.POINTER(i32),
                             ctypes.POINTER(dbl)], i32),
    "gb_batched_plan_tile": ([vp], i32),
    "gb_batched_plan_run": ([vp, vp], i32),
    "gb_batched_plan_destroy": ([vp], i32),
    "gb_batched_plan_info": ([vp, ctypes.POINTER(i64), ctypes.POINTER(i32), ctypes.POINTER(i64),
                              ctypes.POINTER(dbl)], i32),
    "gb_plan_candidates": ([i32, ctypes.POINTER(GbPlan), i32], i32),
    "gb_plan_features": ([i32, i32, i32, i32, i64, i64, ctypes.POINTER(GbPlan), ctypes.POINTER(flt)], i32),
    "gb_plan_set_model": ([ctypes.c_char_p], i32),
    "gb_plan_choose": ([i32, i32, i32, i32, i64, i64, ctypes.POINTER(GbPlan), ctypes.POINTER(dbl)], i32),
    "gb_plan_mixed_candidates": ([i64, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(GbPlan), i32], i32),
    "gb_plan_choose_precision": ([i32, i32, i32, i64, i64, ctypes.POINTER(i32), ctypes.POINTER(i64),
                                  ctypes.POINTER(GbPlan), ctypes.POINTER(dbl)], i32),
    "gb_autotune_time": ([i32, i32, i32, i32, i32, i64, i64, dbl, vp, i64, vp, i64, ctypes.POINTER(GbPlan), i32,
                          i32, ctypes.POINTER(dbl), vp], i32),
    "gb_autotune": ([i32, i32, i32, i32, i32, i64, i64, dbl, vp, i64, vp, i64, ctypes.POINTER(GbPlan),
                     ctypes.POINTER(dbl), vp], i32),
    "gb_mlp_param_count": ([i32], i64),
    "gb_mlp_forward": ([vp, i32, vp, i64, vp, vp, vp], i32),
    "gb_mlp_backward": ([vp, i32, vp, vp, vp, i64, vp, vp], i32),
    "gb_mlp_loss": ([vp, vp, i64, vp, vp, vp], i32),
    "gb_mlp_adam": ([vp, vp, vp, vp, i64, flt, flt, flt, flt, i32, vp], i32),
    "gb_mixed_history": ([ctypes.POINTER(dbl), ctypes.POINTER(i32), i32], i32),
    "gb_bf16_gemm_update": ([i64, i64, i64, vp, i64, vp, i64, vp, i64, flt, vp], i32),
    "gb_device_status": ([i32], i32),
    "gb_kernel_launches": ([], ctypes.c_uint64),
    "gb_profile_enable": ([i32], i32),
    "gb_profile_read": ([i32, ctypes.POINTER(i64), ctypes.POINTER(dbl), ctypes.POINTER(dbl),
                         ctypes.POINTER(dbl)], i32),
}


def lib():
    """Load libgbtrsm.so (raises if it is missing)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
        l = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(l, name)
            f.argtypes = args
            f.restype = res
        _lib = l
    return _lib


def _plan_ptr(plan):
    if plan is None:
        return None
    if isinstance(plan, GbPlan):
        return ctypes.byref(plan)
    d = dict(plan)
    return ctypes.byref(GbPlan(d.get("driver", 0), d.get("nb", 64), d.get("depth", 0), d.get("reserved", 0)))


# ---- one-to-one C entry points ------------------------------------------------

def gb_dtrsm(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream=0):
    return lib().gb_dtrsm(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream or None)


def gb_strsm(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream=0):
    return lib().gb_strsm(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream or None)


def gb_dtrsm_plan(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, plan, stream=0):
    return lib().gb_dtrsm_plan(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb,
                               _plan_ptr(plan), stream or None)


def gb_strsm_plan(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, plan, stream=0):
    return lib().gb_strsm_plan(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb,
                               _plan_ptr(plan), stream or None)


def gb_plan_counts(plan, k):
    nd, ng, nbk, md = i64(), i64(), i64(), dbl()
    st = lib().gb_plan_counts(_plan_ptr(plan), k, ctypes.byref(nd), ctypes.byref(ng),
                              ctypes.byref(nbk), ctypes.byref(md))
    if st != 0:
        raise GbError("gb_plan_counts", st)
    return dict(n_diag=nd.value, n_gemm=ng.value, n_offdiag_blocks=nbk.value,
                gemm_madds_per_col=md.value)


PREC_BF16, PREC_FP8 = 0, 1


def gb_dtrsm_mixed(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, stream=0):
    """Returns (status, iters, est_err)."""
    it, est = i32(), dbl()
    st = lib().gb_dtrsm_mixed(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter,
                              ctypes.byref(it), ctypes.byref(est), stream or None)
    return st, it.value, est.value


def gb_dtrsm_mixed_noalloc(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, stream=0):
    """As gb_dtrsm_mixed, with the library's fixed scratch instead of any
    device allocation.  Returns (status, iters, est_err)."""
    it, est = i32(), dbl()
    st = lib().gb_dtrsm_mixed_noalloc(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter,
                                      ctypes.byref(it), ctypes.byref(est), stream or None)
    return st, it.value, est.value


def gb_dtrsm_mixed_host(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, stream=0):
    """As gb_dtrsm_mixed with A and B in host memory (A and B are host
    addresses; page-locked memory lets the copies overlap computation).
    Returns (status, iters, est_err)."""
    it, est = i32(), dbl()
    st = lib().gb_dtrsm_mixed_host(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter,
                                   ctypes.byref(it), ctypes.byref(est), stream or None)
    return st, it.value, est.value


def gb_mixed_host_bytes(side, uplo, m, n):
    """(host->device, device->host) bytes of one gb_dtrsm_mixed_host call."""
    d2h = i64()
    h2d = lib().gb_mixed_host_bytes(side, uplo, m, n, ctypes.byref(d2h))
    return int(h2d), int(d2h.value)


def gb_dtrsm_mixed_leaf(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, leaf,
                        stream=0):
    """gb_dtrsm_mixed with an explicit leaf order.  Returns (status, iters, est_err)."""
    it, est = i32(), dbl()
    st = lib().gb_dtrsm_mixed_leaf(side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, tol, prec, max_iter, leaf,
                                   ctypes.byref(it), ctypes.byref(est), stream or None)
    return st, it.value, est.value


def gb_set_lookahead(on):
    """Plain solves' lookahead on (1) / off (0); -1 queries.  Returns the previous setting."""
    return lib().gb_set_lookahead(on)


def gb_gemm_update(dtype, M, N, K, A, lda, B, ldb, C, ldc, alpha, stream=0):
    return lib().gb_gemm_update(dtype, M, N, K, A, lda, B, ldb, C, ldc, alpha, stream or None)


def gb_dpotrf(uplo, n, A, lda, stream=0):
    """Returns (status, info)."""
    info = i64()
    st = lib().gb_dpotrf(uplo, n, A, lda, ctypes.byref(info), stream or None)
    return st, info.value


def gb_spotrf(uplo, n, A, lda, stream=0):
    """Returns (status, info)."""
    info = i64()
    st = lib().gb_spotrf(uplo, n, A, lda, ctypes.byref(info), stream or None)
    return st, info.value


def potrf(uplo, A, stream=None):
    """Cholesky factorisation in place on a torch float64 / float32 CUDA
    tensor (column-major, n x n): the named triangle is overwritten by the
    factor.  Returns info (0, or the order of the first leading minor that is
    not positive definite); raises GbError on argument / CUDA errors."""
    import torch
    n = A.shape[0]
    if A.dim() != 2 or A.shape[1] != n:
        raise ValueError("A must be square")
    pa, lda = _colmajor(A, "A")
    s = _stream_handle(stream)
    if A.dtype == torch.float64:
        st, info = gb_dpotrf(uplo, n, pa, lda, s)
        fn = "gb_dpotrf"
    elif A.dtype == torch.float32:
        st, info = gb_spotrf(uplo, n, pa, lda, s)
        fn = "gb_spotrf"
    else:
        raise TypeError(f"unsupported dtype {A.dtype}")
    if st != 0:
        raise GbError(fn, st)
    return info


def gb_mixed_workspace_release(stream=0):
    """Free the mixed solves' cached work space on the current device."""
    return lib().gb_mixed_workspace_release(stream or None)


class _BatchArgs:
    """Host descriptor arrays of a batch (kept alive while in use)."""

    def __init__(self, dtype, items):
        import numpy as np
        c = len(items)
        self.count = c
        self.side = np.array([it["side"] for it in items], dtype=np.int8)
        self.uplo = np.array([it["uplo"] for it in items], dtype=np.int8)
        self.trans = np.array([it["trans"] for it in items], dtype=np.int8)
        self.diag = np.array([it["diag"] for it in items], dtype=np.int8)
        self.m = np.array([it["m"] for it in items], dtype=np.int64)
        self.n = np.array([it["n"] for it in items], dtype=np.int64)
        self.alpha = np.array([it["alpha"] for it in items], dtype=np.float64 if dtype == 0 else np.float32)
        self.A = (ctypes.c_void_p * max(c, 1))(*[it["A_ptr"] for it in items])
        self.B = (ctypes.c_void_p * max(c, 1))(*[it["B_ptr"] for it in items])
        self.lda = np.array([it["lda"] for it in items], dtype=np.int64)
        self.ldb = np.array([it["ldb"] for it in items], dtype=np.int64)

    def args(self):
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        return [self.count, p(self.side), p(self.uplo), p(self.trans), p(self.diag), p(self.m), p(self.n),
                p(self.alpha), ctypes.cast(self.A, ctypes.c_void_p), p(self.lda),
                ctypes.cast(self.B, ctypes.c_void_p), p(self.ldb)]


def gb_trsm_batched(dtype, items, stream=0):
    """items: list of dicts with side, uplo, trans, diag, m, n, alpha, A_ptr,
    lda, B_ptr, ldb (device pointers as ints).  Returns the status."""
    a = _BatchArgs(dtype, items)
    return lib().gb_trsm_batched(dtype, *a.args(), stream or None)


def gb_batched_autotune(dtype, items, reps=3, stream=0):
    """Time the batched kernel's tile shapes on these problems (B restored
    afterwards).  Returns (best tile, [ms with tile 1, ms with tile 2])."""
    a = _BatchArgs(dtype, items)
    tile, ms = i32(), (dbl * 2)()
    st = lib().gb_batched_autotune(dtype, *a.args(), reps, stream or None, ctypes.byref(tile), ms)
    if st != 0:
        raise GbError("gb_batched_autotune", st)
    return tile.value, [ms[0], ms[1]]


class BatchedPlan:
    """gb_batched_plan_* handle (work queue + CUDA graph for fixed pointers);
    tile = rows per thread of the kernel's gemm tasks (1 or 2; 0 = default)."""

    def __init__(self, dtype, items, stream=0, tile=0):
        self._args = _BatchArgs(dtype, items)
        h = vp()
        st = lib().gb_batched_plan_create_tiled(dtype, *self._args.args(), tile, stream or None, ctypes.byref(h))
        if st != 0:
            raise GbError("gb_batched_plan_create_tiled", st)
        self.handle = h
        self.tile = lib().gb_batched_plan_tile(h)

    def run(self, stream=0):
        st = lib().gb_batched_plan_run(self.handle, stream or None)
        if st != 0:
            raise GbError("gb_batched_plan_run", st)

    def info(self):
        u, g, big, fl = i64(), i32(), i64(), dbl()
        lib().gb_batched_plan_info(self.handle, ctypes.byref(u), ctypes.byref(g), ctypes.byref(big),
                                   ctypes.byref(fl))
        return dict(units=u.value, grid=g.value, large_instances=big.value, flops=fl.value)

    def close(self):
        if self.handle:
            lib().gb_batched_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gb_plan_candidates(dtype=0):
    arr = (GbPlan * 64)()
    n = lib().gb_plan_candidates(dtype, arr, 64)
    return [dict(driver=arr[i].driver, nb=arr[i].nb, depth=arr[i].depth) for i in range(n)]


N_FEATURES = 17


def gb_plan_features(dtype, side, uplo, trans, m, n, plan):
    f = (flt * N_FEATURES)()
    lib().gb_plan_features(dtype, side, uplo, trans, m, n, _plan_ptr(plan), f)
    return list(f)


def gb_plan_set_model(path):
    return lib().gb_plan_set_model(None if path is None else str(path).encode())


def gb_plan_choose(dtype, side, uplo, trans, m, n):
    p, ms = GbPlan(), dbl()
    st = lib().gb_plan_choose(dtype, side, uplo, trans, m, n, ctypes.byref(p), ctypes.byref(ms))
    return st, dict(driver=p.driver, nb=p.nb, depth=p.depth), ms.value


def gb_plan_mixed_candidates(k):
    """[(prec, leaf, plan dict), ...] of the precision decision for order k."""
    prec = (i32 * 8)()
    leaf = (i64 * 8)()
    plans = (GbPlan * 8)()
    n = lib().gb_plan_mixed_candidates(k, prec, leaf, plans, 8)
    return [(prec[i], leaf[i], dict(driver=plans[i].driver, nb=plans[i].nb, depth=plans[i].depth))
            for i in range(n)]


def gb_plan_choose_precision(side, uplo, trans, m, n):
    """(status, prec (-1 = plain FP64), leaf, plan dict, predicted ms)."""
    pr, lf, p, ms = i32(), i64(), GbPlan(), dbl()
    st = lib().gb_plan_choose_precision(side, uplo, trans, m, n, ctypes.byref(pr), ctypes.byref(lf),
                                        ctypes.byref(p), ctypes.byref(ms))
    return st, pr.value, lf.value, dict(driver=p.driver, nb=p.nb, depth=p.depth), ms.value


def gb_autotune_time(dtype, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, plans, reps=2, stream=0):
    arr = (GbPlan * len(plans))(*[GbPlan(p["driver"], p["nb"], p["depth"], 0) for p in plans])
    out = (dbl * len(plans))()
    st = lib().gb_autotune_time(dtype, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, arr, len(plans),
                                reps, out, stream or None)
    if st != 0:
        raise GbError("gb_autotune_time", st)
    return list(out)


def gb_autotune(dtype, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, stream=0):
    p, ms = GbPlan(), dbl()
    st = lib().gb_autotune(dtype, side, uplo, trans, diag, m, n, alpha, A, lda, B, ldb, ctypes.byref(p),
                           ctypes.byref(ms), stream or None)
    if st != 0:
        raise GbError("gb_autotune", st)
    return dict(driver=p.driver, nb=p.nb, depth=p.depth), ms.value


def gb_mlp_param_count(in_dim):
    return lib().gb_mlp_param_count(in_dim)


def gb_mlp_forward(params, in_dim, X, n, Y, Z=0, stream=0):
    return lib().gb_mlp_forward(params, in_dim, X, n, Y, Z or None, stream or None)


def gb_mlp_backward(params, in_dim, X, Z, dY, n, grads, stream=0):
    return lib().gb_mlp_backward(params, in_dim, X, Z, dY, n, grads, stream or None)


def gb_mlp_loss(Y, T, n, dY, loss=0, stream=0):
    return lib().gb_mlp_loss(Y, T, n, dY, loss or None, stream or None)


def gb_mlp_adam(params, grads, m, v, np_, lr, beta1, beta2, eps, step, stream=0):
    return lib().gb_mlp_adam(params, grads, m, v, np_, lr, beta1, beta2, eps, step, stream or None)


def gb_mixed_history(cap=64):
    """[(rho_t, levels_t), ...] of the last mixed solve on this thread."""
    rho = (dbl * cap)()
    lev = (i32 * cap)()
    n = lib().gb_mixed_history(rho, lev, cap)
    return [(rho[i], lev[i]) for i in range(min(n, cap))]


def trsm_mixed(side, uplo, trans, diag, alpha, A, B, tol=1e-11, prec=0, max_iter=30, stream=None):
    """Mixed-precision solve on torch float64 CUDA tensors (column-major), in
    place on B.  Returns (status, iters, est_err); raises on argument / CUDA
    errors (status < 0 or == STATUS_CUDA_ERROR)."""
    m, n = B.shape
    pa, lda = _colmajor(A, "A")
    pb, ldb = _colmajor(B, "B")
    st, it, est = gb_dtrsm_mixed(side, uplo, trans, diag, m, n, float(alpha), pa, lda, pb, ldb, float(tol),
                                 prec, max_iter, _stream_handle(stream))
    if st < 0 or st in (STATUS_CUDA_ERROR, STATUS_TIMEOUT):
        raise GbError("gb_dtrsm_mixed", st)
    return st, it, est


def trsm_mixed_host(side, uplo, trans, diag, alpha, A, B, tol=1e-11, prec=0, max_iter=30, stream=None):
    """Mixed-precision solve on torch float64 CPU tensors (column-major; pin
    them for overlapped copies), in place on B.  Returns (status, iters,
    est_err); raises on argument / CUDA errors."""
    if A.device.type != "cpu" or B.device.type != "cpu":
        raise ValueError("trsm_mixed_host takes host (CPU) tensors")
    m, n = B.shape
    pa, lda = _colmajor(A, "A")
    pb, ldb = _colmajor(B, "B")
    st, it, est = gb_dtrsm_mixed_host(side, uplo, trans, diag, m, n, float(alpha), pa, lda, pb, ldb, float(tol),
                                      prec, max_iter, _stream_handle(stream))
    if st < 0 or st in (STATUS_CUDA_ERROR, STATUS_TIMEOUT):
        raise GbError("gb_dtrsm_mixed_host", st)
    return st, it, est


def gb_bf16_gemm_update(M, N, K, A, lda, B, ldb, C, ldc, alpha, stream=0):
    return lib().gb_bf16_gemm_update(M, N, K, A, lda, B, ldb, C, ldc, alpha, stream or None)


def gb_device_status(clear=1):
    return lib().gb_device_status(clear)


def gb_status_string(status):
    return lib().gb_status_string(status).decode()


status_string = gb_status_string


def gb_last_cuda_error():
    return lib().gb_last_cuda_error()


def gb_version():
    return lib().gb_version()


KERNEL_KINDS = ["diag", "gemm_simt", "gemm_tc", "residual", "convert", "batched", "mlp", "graph"]


def gb_kernel_launches():
    return lib().gb_kernel_launches()


def gb_profile_enable(on):
    return lib().gb_profile_enable(int(bool(on)))


def gb_profile_read(kind):
    n, ms, fl, by = i64(), dbl(), dbl(), dbl()
    st = lib().gb_profile_read(kind, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl), ctypes.byref(by))
    if st != 0:
        raise GbError("gb_profile_read", st)
    return dict(launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value)


# ---- torch-tensor conveniences ---------------------------------------------------

def _colmajor(t, name):
    if t.dim() != 2:
        raise ValueError(f"{name} must be 2-D")
    if t.numel() > 0 and t.stride(0) != 1 and t.shape[0] > 1:
        raise ValueError(f"{name} must be column-major (stride(0) == 1)")
    return t.data_ptr(), max(1, t.stride(1) if t.shape[1] > 1 else t.shape[0])


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def trsm(side, uplo, trans, diag, alpha, A, B, plan=None, stream=None):
    """Solve in place on torch CUDA tensors (float64 or float32, column-major).

    B (m x n) is overwritten by X.  Raises GbError on a nonzero status.
    """
    import torch
    m, n = B.shape
    pa, lda = _colmajor(A, "A")
    pb, ldb = _colmajor(B, "B")
    s = _stream_handle(stream)
    if B.dtype == torch.float64:
        st = gb_dtrsm_plan(side, uplo, trans, diag, m, n, float(alpha), pa, lda, pb, ldb, plan, s)
        fn = "gb_dtrsm_plan"
    elif B.dtype == torch.float32:
        st = gb_strsm_plan(side, uplo, trans, diag, m, n, float(alpha), pa, lda, pb, ldb, plan, s)
        fn = "gb_strsm_plan"
    else:
        raise TypeError(f"unsupported dtype {B.dtype}")
    if st != 0:
        raise GbError(fn, st)
    return B


def colmajor_empty(m, n, dtype, device="cuda"):
    """An m x n column-major torch tensor (a transposed row-major buffer)."""
    import torch
    return torch.empty((n, m), dtype=dtype, device=device).t()


def to_device_colmajor(x, dtype=None, device="cuda"):
    """Copy a numpy/torch 2-D array to a column-major CUDA tensor."""
    import numpy as np
    import torch
    t = torch.as_tensor(np.asarray(x)) if not isinstance(x, torch.Tensor) else x
    if dtype is not None:
        t = t.to(dtype)
    out = colmajor_empty(t.shape[0], t.shape[1], t.dtype, device)
    out.copy_(t)
    return out
