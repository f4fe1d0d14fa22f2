"""Python binding of libkes (include/kes.h): the filtered time-domain Krylov
eigensolver of Nannen & Wess (arXiv:2402.08515) on GB300.

Argument marshalling only: every step of the method runs in the CUDA library.
Functions keep the C names (``kes_create``, ``kes_filter_apply``, ...) and
take numpy arrays (host) or torch CUDA tensors (device); a ``KesError`` is
raised for every non-OK status except KES_INFO_INVARIANT_SUBSPACE, which is
reported in the result. There is no CPU fallback: importing this package
without a built ``libkes.so`` raises ImportError.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import weakref

import numpy as np

__all__ = [
    "KesError", "KesOpts", "KesSolveOpts", "KesResult", "KesStats", "lib", "LIB_PATH",
    "KES_PREC_FP64", "KES_PREC_FP32", "KES_MEM_DEVICE", "KES_MEM_HOST", "KES_STEPPER_LEAPFROG",
    "KES_STEPPER_LEAPFROG4", "KES_REFINE_FP64", "KES_REFINE_F32X2",
    "kes_opts_default", "kes_solve_opts_default", "kes_strerror", "kes_create", "kes_destroy",
    "kes_size", "kes_sync", "kes_estimate_omega_max", "kes_set_filter", "kes_set_filters",
    "kes_alpha_table", "kes_filter_response", "kes_sym_eig", "kes_step_bytes",
    "kes_filter_apply", "kes_krylov_solve", "kes_get_stats", "kes_reset_stats",
    "Context", "header_functions", "kes_filter_apply_noalloc", "KES_NOALLOC_MAX_N",
    "kes_create_batch", "kes_mesh_count", "kes_estimate_omega_max_batch", "kes_set_filters_batch",
    "kes_block_krylov_solve", "kes_set_weights", "kes_alpha_gaussian", "kes_filter_apply_columns",
    "kes_alpha_triangle", "kes_weights_response", "kes_launch_shapes", "kes_subspace_solve",
]

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libkes.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "kes.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2402_08515_gb300/build.py` "
                      "(no CPU fallback exists)")
lib = C.CDLL(LIB_PATH)

KES_OK, KES_INFO_INVARIANT_SUBSPACE = 0, 1
KES_PREC_FP64, KES_PREC_FP32 = 0, 1
KES_MEM_DEVICE, KES_MEM_HOST = 0, 1
KES_STEPPER_LEAPFROG, KES_STEPPER_LEAPFROG4 = 0, 1
KES_REFINE_FP64, KES_REFINE_F32X2 = 0, 1


class KesError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {lib.kes_strerror(status).decode()} (status {status})")


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class KesOpts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("sell_sigma", C.c_int32), ("use_graph", C.c_int32),
                ("block_b", C.c_int32), ("autotune", C.c_int32), ("step_variant", C.c_int32),
                ("stream", C.c_void_p), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_user", C.c_void_p), ("stepper", C.c_int32), ("blk_variant", C.c_int32),
                ("compact_cols", C.c_int32)]


class KesSolveOpts(C.Structure):
    _fields_ = [("kmax", C.c_int32), ("check_every", C.c_int32), ("n_wanted", C.c_int32),
                ("want_vectors", C.c_int32), ("tol", C.c_double), ("refine_sweeps", C.c_int32),
                ("refine_L", C.c_int32), ("refine_extra", C.c_int32), ("refine_precision", C.c_int32)]


class KesResult(C.Structure):
    _fields_ = [("n", C.c_int64), ("n_pairs", C.c_int32), ("k_used", C.c_int32), ("breakdown", C.c_int32),
                ("n_ritz", C.c_int32), ("time_steps", C.c_int64), ("omega2", C.POINTER(C.c_double)),
                ("omega", C.POINTER(C.c_double)), ("rel_res", C.POINTER(C.c_double)),
                ("abs_res", C.POINTER(C.c_double)), ("vectors", C.POINTER(C.c_double)),
                ("ritz_omega2", C.POINTER(C.c_double)), ("ritz_rel_res", C.POINTER(C.c_double)),
                ("solve_ms", C.c_double), ("refine_steps", C.c_int64),
                ("interval", C.POINTER(C.c_int32))]


class KesStats(C.Structure):
    _fields_ = [("filter_calls", C.c_int64), ("filter_steps", C.c_int64), ("kernel_launches", C.c_int64),
                ("filter_ms", C.c_double), ("solve_other_ms", C.c_double), ("bytes_per_step", C.c_int64),
                ("step_variant", C.c_int32), ("step_grid", C.c_int32), ("blk_variant", C.c_int32),
                ("blk_grid", C.c_int32)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_sig = {
    "kes_opts_default": (None, [C.POINTER(KesOpts)]),
    "kes_solve_opts_default": (None, [C.POINTER(KesSolveOpts)]),
    "kes_strerror": (C.c_char_p, [C.c_int32]),
    "kes_create": (C.c_int, [C.POINTER(_P), C.c_int64, _P, _P, _P, _P, C.POINTER(KesOpts)]),
    "kes_destroy": (None, [_P]),
    "kes_size": (C.c_int64, [_P]),
    "kes_sync": (C.c_int, [_P]),
    "kes_estimate_omega_max": (C.c_int, [_P, C.c_int32, _P, _D, _D]),
    "kes_set_filter": (C.c_int, [_P, C.c_double, C.c_double, C.c_double, C.c_int32]),
    "kes_set_filters": (C.c_int, [_P, C.c_int32, _P, _P, C.c_double, C.c_int32]),
    "kes_alpha_table": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int32, _P]),
    "kes_filter_response": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int32, _P, C.c_int64, _P]),
    "kes_sym_eig": (C.c_int, [C.c_int32, _P, _P, _P]),
    "kes_step_bytes": (C.c_int64, [_P, C.c_int32, C.c_int32]),
    "kes_filter_apply": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32]),
    "kes_filter_apply_columns": (C.c_int, [_P, _P, _P, C.c_int32, C.c_int32]),
    "kes_krylov_solve": (C.c_int, [_P, _P, C.c_int32, C.POINTER(KesSolveOpts), C.POINTER(C.POINTER(KesResult))]),
    "kes_result_free": (None, [C.POINTER(KesResult)]),
    "kes_get_stats": (C.c_int, [_P, C.POINTER(KesStats)]),
    "kes_reset_stats": (C.c_int, [_P]),
    "kes_filter_apply_noalloc": (C.c_int, [C.c_int64, _P, _P, _P, _P, _P, C.c_int32, _P, _P, _P]),
    "kes_create_batch": (C.c_int, [C.POINTER(_P), C.c_int32, _P, _P, _P, _P, _P, C.POINTER(KesOpts)]),
    "kes_mesh_count": (C.c_int32, [_P]),
    "kes_estimate_omega_max_batch": (C.c_int, [_P, C.c_int32, _P, _P, _P]),
    "kes_set_filters_batch": (C.c_int, [_P, C.c_int32, _P, _P, _P, C.c_int32]),
    "kes_block_krylov_solve": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.POINTER(KesSolveOpts),
                                         C.POINTER(C.POINTER(KesResult))]),
    "kes_subspace_solve": (C.c_int, [_P, _P, C.c_int32, C.c_int32, C.POINTER(KesSolveOpts),
                                         C.POINTER(C.POINTER(KesResult))]),
    "kes_set_weights": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P, C.c_int32]),
    "kes_alpha_gaussian": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int32, _P]),
    "kes_alpha_triangle": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_int32, _P]),
    "kes_weights_response": (C.c_int, [_P, C.c_double, C.c_int32, _P, C.c_int64, _P]),
    "kes_launch_shapes": (None, [C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def header_functions(path: str = HEADER) -> list[str]:
    """Names of every function declared in include/kes.h."""
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(kes_[a-z0-9_]+)\s*\(", text)))


def _check(status: int, where: str, allow_info: bool = False) -> int:
    if status == KES_OK or (allow_info and status == KES_INFO_INVARIANT_SUBSPACE):
        return status
    raise KesError(status, where)


def _f64_host(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


# ------------------------------------------------------------------ C names

def kes_opts_default() -> KesOpts:
    o = KesOpts()
    lib.kes_opts_default(C.byref(o))
    return o


def kes_solve_opts_default() -> KesSolveOpts:
    o = KesSolveOpts()
    lib.kes_solve_opts_default(C.byref(o))
    return o


def kes_strerror(status: int) -> str:
    return lib.kes_strerror(status).decode()


def kes_create(n, row_ptr, col, val, m_diag, opts: KesOpts | None = None) -> int:
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = _f64_host(val)
    m_diag = _f64_host(m_diag)
    h = C.c_void_p()
    _check(lib.kes_create(C.byref(h), int(n), _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(m_diag),
                          C.byref(opts) if opts is not None else None), "kes_create")
    return h.value


def kes_destroy(ctx: int) -> None:
    lib.kes_destroy(ctx)


def kes_size(ctx: int) -> int:
    return lib.kes_size(ctx)


def kes_sync(ctx: int) -> None:
    _check(lib.kes_sync(ctx), "kes_sync")


def kes_estimate_omega_max(ctx: int, iters: int, v0) -> tuple[float, float]:
    v0 = _f64_host(v0)
    om, g = C.c_double(), C.c_double()
    _check(lib.kes_estimate_omega_max(ctx, int(iters), _ptr(v0), C.byref(om), C.byref(g)), "kes_estimate_omega_max")
    return om.value, g.value


def kes_set_filter(ctx: int, omega_min: float, omega_max: float, tau: float, L: int) -> None:
    _check(lib.kes_set_filter(ctx, float(omega_min), float(omega_max), float(tau), int(L)), "kes_set_filter")


def kes_set_filters(ctx: int, omega_min, omega_max, tau: float, L: int) -> None:
    a, b = _f64_host(omega_min), _f64_host(omega_max)
    _check(lib.kes_set_filters(ctx, len(a), _ptr(a), _ptr(b), float(tau), int(L)), "kes_set_filters")


def kes_alpha_table(omega_min: float, omega_max: float, tau: float, L: int) -> np.ndarray:
    out = np.empty(L + 1)
    _check(lib.kes_alpha_table(float(omega_min), float(omega_max), float(tau), int(L), _ptr(out)),
           "kes_alpha_table")
    return out


def kes_filter_response(omega_min: float, omega_max: float, tau: float, L: int, omega) -> np.ndarray:
    omega = _f64_host(np.atleast_1d(omega))
    out = np.empty_like(omega)
    _check(lib.kes_filter_response(float(omega_min), float(omega_max), float(tau), int(L), _ptr(omega),
                                   omega.size, _ptr(out)), "kes_filter_response")
    return out


def kes_launch_shapes() -> tuple:
    """(launch shapes of the single-vector step kernel, of the block step kernel)."""
    a, b = C.c_int32(), C.c_int32()
    lib.kes_launch_shapes(C.byref(a), C.byref(b))
    return a.value, b.value


def kes_weights_response(alpha, tau: float, omega) -> np.ndarray:
    """beta~(omega) of the weight table alpha[0..L]."""
    alpha = _f64_host(alpha)
    omega = _f64_host(np.atleast_1d(omega))
    out = np.empty_like(omega)
    _check(lib.kes_weights_response(_ptr(alpha), float(tau), alpha.size - 1, _ptr(omega), omega.size, _ptr(out)),
           "kes_weights_response")
    return out


def kes_alpha_gaussian(center: float, sigma: float, tau: float, L: int) -> np.ndarray:
    out = np.empty(L + 1)
    _check(lib.kes_alpha_gaussian(float(center), float(sigma), float(tau), int(L), _ptr(out)), "kes_alpha_gaussian")
    return out


def kes_alpha_triangle(center: float, half_width: float, tau: float, L: int) -> np.ndarray:
    out = np.empty(L + 1)
    _check(lib.kes_alpha_triangle(float(center), float(half_width), float(tau), int(L), _ptr(out)),
           "kes_alpha_triangle")
    return out


def kes_set_weights(ctx: int, alpha, omega_min, omega_max, tau, L: int) -> None:
    """alpha: (n_mesh, F, L+1) weight tables; omega_min/omega_max: (n_mesh, F); tau: (n_mesh,)."""
    a = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64).reshape(-1))
    wmin = np.ascontiguousarray(np.atleast_2d(omega_min), dtype=np.float64)
    wmax = np.ascontiguousarray(np.atleast_2d(omega_max), dtype=np.float64)
    t = _f64_host(np.atleast_1d(tau))
    F = wmin.shape[1]
    if a.size != wmin.shape[0] * F * (L + 1):
        raise ValueError("alpha must hold n_mesh * F * (L + 1) weights")
    _check(lib.kes_set_weights(ctx, F, a.ctypes.data, wmin.ctypes.data, wmax.ctypes.data, t.ctypes.data, int(L)),
           "kes_set_weights")


def kes_sym_eig(A) -> tuple[np.ndarray, np.ndarray]:
    A = np.asfortranarray(A, dtype=np.float64)
    k = A.shape[0]
    w = np.empty(k)
    V = np.empty((k, k), order="F")
    _check(lib.kes_sym_eig(k, A.ctypes.data, w.ctypes.data, V.ctypes.data), "kes_sym_eig")
    return w, V


def kes_step_bytes(ctx: int, b: int = 1, F: int = 1) -> int:
    return lib.kes_step_bytes(ctx, int(b), int(F))


def kes_filter_apply(ctx: int, r_in, r_out, b: int = 1) -> None:
    """r_in: (b, n) float64, r_out: (F, b, n) float64; both numpy (host) or both CUDA tensors."""
    dev = _is_device(r_in)
    if dev != _is_device(r_out):
        raise ValueError("r_in and r_out must both be host arrays or both device tensors")
    if not dev:
        if not (isinstance(r_out, np.ndarray) and r_out.dtype == np.float64 and r_out.flags.c_contiguous):
            raise ValueError("r_out must be a C-contiguous float64 numpy array")
        r_in = _f64_host(r_in)
    _check(lib.kes_filter_apply(ctx, _ptr(r_in), _ptr(r_out), int(b), KES_MEM_DEVICE if dev else KES_MEM_HOST),
           "kes_filter_apply")


def kes_filter_apply_columns(ctx: int, r_in, r_out, b: int) -> None:
    """r_in, r_out: (b, n) float64, both numpy (host) or both CUDA tensors; column j is
    filtered with weight table j // (b // F)."""
    dev = _is_device(r_in)
    if dev != _is_device(r_out):
        raise ValueError("r_in and r_out must both be host arrays or both device tensors")
    if not dev:
        if not (isinstance(r_out, np.ndarray) and r_out.dtype == np.float64 and r_out.flags.c_contiguous):
            raise ValueError("r_out must be a C-contiguous float64 numpy array")
        r_in = _f64_host(r_in)
    _check(lib.kes_filter_apply_columns(ctx, _ptr(r_in), _ptr(r_out), int(b),
                                        KES_MEM_DEVICE if dev else KES_MEM_HOST), "kes_filter_apply_columns")


def _arr(p, k):
    return np.ctypeslib.as_array(p, shape=(k,)).copy() if k > 0 else np.zeros(0)


def _result_dict(rp, st) -> dict:
    """The result as a dict of numpy arrays. The small arrays are copied; the Ritz vectors
    (often gigabytes) are not: their array views the library's buffer, and the result is
    released when that array is garbage collected (or at once when there are none)."""
    r = rp.contents
    keep = False
    try:
        p = r.n_pairs
        out = dict(status=st, n=r.n, n_pairs=p, k_used=r.k_used, breakdown=bool(r.breakdown),
                   time_steps=r.time_steps, omega2=_arr(r.omega2, p), omega=_arr(r.omega, p),
                   rel_res=_arr(r.rel_res, p), abs_res=_arr(r.abs_res, p),
                   ritz_omega2=_arr(r.ritz_omega2, r.n_ritz), ritz_rel_res=_arr(r.ritz_rel_res, r.n_ritz),
                   solve_ms=r.solve_ms, refine_steps=r.refine_steps, vectors=None,
                   interval=(np.ctypeslib.as_array(r.interval, shape=(p,)).astype(np.int64) if p > 0
                             else np.zeros(0, dtype=np.int64)))
        if r.vectors and p > 0:
            flat = np.ctypeslib.as_array(r.vectors, shape=(p * r.n,))
            weakref.finalize(flat, lib.kes_result_free, rp)
            keep = True
            out["vectors"] = flat.reshape(p, r.n)
    finally:
        if not keep:
            lib.kes_result_free(rp)
    return out


def kes_krylov_solve(ctx: int, r0, sopts: KesSolveOpts | None = None) -> dict:
    dev = _is_device(r0)
    if not dev:
        r0 = _f64_host(r0)
    rp = C.POINTER(KesResult)()
    st = lib.kes_krylov_solve(ctx, _ptr(r0), KES_MEM_DEVICE if dev else KES_MEM_HOST,
                              C.byref(sopts) if sopts is not None else None, C.byref(rp))
    _check(st, "kes_krylov_solve", allow_info=True)
    return _result_dict(rp, st)


def kes_block_krylov_solve(ctx: int, R0, b: int, sopts: KesSolveOpts | None = None) -> list[dict]:
    """R0: (b, n_total) start vectors (numpy or CUDA tensor); one result dict per mesh."""
    dev = _is_device(R0)
    if not dev:
        R0 = _f64_host(R0)
    nm = lib.kes_mesh_count(ctx)
    arr = (C.POINTER(KesResult) * nm)()
    st = lib.kes_block_krylov_solve(ctx, _ptr(R0), int(b), KES_MEM_DEVICE if dev else KES_MEM_HOST,
                                    C.byref(sopts) if sopts is not None else None,
                                    C.cast(arr, C.POINTER(C.POINTER(KesResult))))
    _check(st, "kes_block_krylov_solve", allow_info=True)
    return [_result_dict(arr[j], st) for j in range(nm)]


def kes_subspace_solve(ctx: int, X0, sopts: KesSolveOpts) -> list[dict]:
    """X0: (p, n_total) start vectors (numpy or CUDA tensor); one result dict per mesh."""
    dev = _is_device(X0)
    if not dev:
        X0 = _f64_host(X0)
    nm = lib.kes_mesh_count(ctx)
    arr = (C.POINTER(KesResult) * nm)()
    st = lib.kes_subspace_solve(ctx, _ptr(X0), int(X0.shape[0]), KES_MEM_DEVICE if dev else KES_MEM_HOST,
                                C.byref(sopts), C.cast(arr, C.POINTER(C.POINTER(KesResult))))
    _check(st, "kes_subspace_solve", allow_info=True)
    return [_result_dict(arr[j], st) for j in range(nm)]


def kes_mesh_count(ctx: int) -> int:
    return lib.kes_mesh_count(ctx)


def kes_create_batch(problems, opts: KesOpts | None = None) -> int:
    """problems: sequence of objects with n, row_ptr, col, val, m (host arrays)."""
    keep = []
    nm = len(problems)
    n = np.array([p.n for p in problems], dtype=np.int64)
    ptrs = {k: (C.c_void_p * nm)() for k in ("row_ptr", "col", "val", "m")}
    for j, p in enumerate(problems):
        arrs = dict(row_ptr=np.ascontiguousarray(p.row_ptr, dtype=np.int64),
                    col=np.ascontiguousarray(p.col, dtype=np.int32), val=_f64_host(p.val), m=_f64_host(p.m))
        keep.append(arrs)
        for k, a in arrs.items():
            ptrs[k][j] = a.ctypes.data
    h = C.c_void_p()
    _check(lib.kes_create_batch(C.byref(h), nm, n.ctypes.data, C.cast(ptrs["row_ptr"], C.c_void_p),
                                C.cast(ptrs["col"], C.c_void_p), C.cast(ptrs["val"], C.c_void_p),
                                C.cast(ptrs["m"], C.c_void_p), C.byref(opts) if opts is not None else None),
           "kes_create_batch")
    return h.value


def kes_estimate_omega_max_batch(ctx: int, iters: int, v0) -> tuple[np.ndarray, np.ndarray]:
    v0 = _f64_host(v0)
    nm = lib.kes_mesh_count(ctx)
    om, g = np.zeros(nm), np.zeros(nm)
    _check(lib.kes_estimate_omega_max_batch(ctx, int(iters), _ptr(v0), om.ctypes.data, g.ctypes.data),
           "kes_estimate_omega_max_batch")
    return om, g


def kes_set_filters_batch(ctx: int, omega_min, omega_max, tau, L: int) -> None:
    """omega_min/omega_max: (n_mesh, F); tau: (n_mesh,)."""
    a = np.ascontiguousarray(np.atleast_2d(omega_min), dtype=np.float64)
    b = np.ascontiguousarray(np.atleast_2d(omega_max), dtype=np.float64)
    t = _f64_host(np.atleast_1d(tau))
    _check(lib.kes_set_filters_batch(ctx, a.shape[1], a.ctypes.data, b.ctypes.data, t.ctypes.data, int(L)),
           "kes_set_filters_batch")


def kes_get_stats(ctx: int) -> dict:
    s = KesStats()
    _check(lib.kes_get_stats(ctx, C.byref(s)), "kes_get_stats")
    return {name: getattr(s, name) for name, _ in KesStats._fields_}


def kes_reset_stats(ctx: int) -> None:
    _check(lib.kes_reset_stats(ctx), "kes_reset_stats")


KES_NOALLOC_MAX_N = 1048576


def kes_filter_apply_noalloc(n, row_ptr, col, val, tau2m, alpha, L, r_in, r_out, stream=None) -> None:
    """Allocation-free FP64 filter of one vector; every array argument is a CUDA tensor the
    caller owns (int64 row_ptr, int32 col, float64 val / tau2m / alpha / r_in / r_out), all
    contiguous and on one device, which this call makes current. Shapes and dtypes are
    checked here (KesError KES_ERR_ARG otherwise); the CSR contents are not (see kes.h)."""
    import torch
    n, L = int(n), int(L)
    want = {"row_ptr": (row_ptr, torch.int64, n + 1), "col": (col, torch.int32, None),
            "val": (val, torch.float64, None), "tau2m": (tau2m, torch.float64, n),
            "alpha": (alpha, torch.float64, L + 1), "r_in": (r_in, torch.float64, n),
            "r_out": (r_out, torch.float64, n)}
    if 1 <= n <= KES_NOALLOC_MAX_N and L >= 1:
        devs = set()
        for name, (t, dt, size) in want.items():
            if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()
                    and t.dim() == 1 and (size is None or t.numel() == size)):
                raise KesError(-1, f"kes_filter_apply_noalloc: {name} must be a contiguous 1-D CUDA {dt} tensor"
                               + (f" of {size} entries" if size is not None else ""))
            devs.add(t.device)
        if len(devs) != 1 or col.numel() != val.numel():
            raise KesError(-1, "kes_filter_apply_noalloc: tensors on several devices, or col and val differ in length")
        torch.cuda.set_device(devs.pop())
    _check(lib.kes_filter_apply_noalloc(n, _ptr(row_ptr), _ptr(col), _ptr(val), _ptr(tau2m), _ptr(alpha),
                                        L, _ptr(r_in), _ptr(r_out), stream), "kes_filter_apply_noalloc")


# ------------------------------------------------------------------ convenience

class Context:
    """Owns a kes context; device memory through torch's caching allocator when
    ``torch_alloc`` is set, launches on ``stream`` (a torch.cuda.Stream or None)."""

    def __init__(self, problem, precision: str = "fp64", sell_sigma: int = 1, use_graph: bool = True,
                 block_b: int = 1, stream=None, torch_alloc: bool = False, autotune: bool = True,
                 step_variant: int | None = None, stepper: str = "leapfrog", blk_variant: int | None = None,
                 compact_cols: bool = True):
        o = kes_opts_default()
        o.compact_cols = 1 if compact_cols else 0
        o.stepper = {"leapfrog": KES_STEPPER_LEAPFROG, "leapfrog4": KES_STEPPER_LEAPFROG4}[stepper]
        o.autotune = 1 if (autotune and step_variant is None and blk_variant is None) else 0
        o.step_variant = step_variant or 0
        o.blk_variant = blk_variant or 0
        o.precision = KES_PREC_FP32 if precision == "fp32" else KES_PREC_FP64
        o.sell_sigma = sell_sigma
        o.use_graph = 1 if use_graph else 0
        o.block_b = block_b
        if stream is not None:
            o.stream = stream.cuda_stream
        self._keep = []
        if torch_alloc:
            import torch
            dev = torch.cuda.current_device()
            st = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream

            def _alloc(nbytes, user):
                return torch.cuda.caching_allocator_alloc(nbytes, dev, st)

            def _free(ptr, nbytes, user):
                torch.cuda.caching_allocator_delete(ptr)
            a, f = ALLOC_FN(_alloc), FREE_FN(_free)
            self._keep += [a, f]
            o.dev_alloc, o.dev_free = a, f
        if isinstance(problem, (list, tuple)):
            self.n = sum(p.n for p in problem)
            self.handle = kes_create_batch(problem, o)
        else:
            self.n = problem.n
            self.handle = kes_create(problem.n, problem.row_ptr, problem.col, problem.val, problem.m, o)

    def close(self):
        if getattr(self, "handle", None):
            kes_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
