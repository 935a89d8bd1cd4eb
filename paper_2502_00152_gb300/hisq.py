"""Thin Python binding of the C ABI in include/hisq.h (argument marshalling only).

Every function has the name of the C entry point it calls.  Host fields are
numpy complex128 arrays shaped (V, 3) (or (nrhs, V, 3)) in the layout
s = x + X*(y + Y*(z + Z*t)); links are complex128 arrays shaped (V, 4, 3, 3).
Device variants take torch CUDA tensors (complex128 or float64 views of the same
layout) and run on the context's stream.

There is no fallback: if libhisq.so is missing or fails to load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# HISQ_LIBRARY selects another build of the library (e.g. the bounds-checking one)
LIB_PATH = os.environ.get("HISQ_LIBRARY") or os.path.join(_HERE, "libhisq.so")

HISQ_OK = 0
HISQ_ERR_INVALID_ARG = 1
HISQ_ERR_CUDA = 2
HISQ_ERR_OOM = 3
HISQ_ERR_NOT_CONVERGED = 4
HISQ_ERR_NUMERICAL = 5
HISQ_ERR_TIMEOUT = 6
HISQ_ERR_STATE = 7

# storage precisions (hisq_precision)
HISQ_PREC_DOUBLE = 64
HISQ_PREC_SINGLE = 32
HISQ_PREC_HALF = 16
HISQ_PREC_BF16 = 15  # eigenvector storage only
HISQ_PREC_HALF_EV = 14  # FP16 of v * 2^e (4^e >= 3 Vh), 12 B per site; eigenvector storage only
HISQ_PREC_DF64 = 48  # double-float (FP32 hi + lo) reliable-update residuals and test operators


class HisqError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"hisq status {status}: {message}")
        self.status = status


class hisq_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("max_iter", ctypes.c_int), ("precision_sloppy", ctypes.c_int),
                ("link_precision_sloppy", ctypes.c_int), ("delta_rd", ctypes.c_double), ("deflate", ctypes.c_int),
                ("n_defl", ctypes.c_int), ("delta_tr", ctypes.c_double), ("compute_full_residual", ctypes.c_int),
                ("batch", ctypes.c_int), ("guess", ctypes.c_int), ("precision_reliable", ctypes.c_int),
                ("persistent", ctypes.c_int)]


class hisq_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("reliable_updates", ctypes.c_int), ("redeflations", ctypes.c_int),
                ("converged", ctypes.c_int), ("even_residual", ctypes.c_double), ("full_residual", ctypes.c_double),
                ("seconds_total", ctypes.c_double), ("seconds_deflate", ctypes.c_double),
                ("seconds_dslash_oe", ctypes.c_double), ("seconds_dslash_eo", ctypes.c_double),
                ("profiled_iterations", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class hisq_eig_params(ctypes.Structure):
    _fields_ = [("n_ev", ctypes.c_int), ("n_kr", ctypes.c_int), ("n_keep", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_restarts", ctypes.c_int), ("cheby_degree", ctypes.c_int), ("a_min", ctypes.c_double),
                ("a_max", ctypes.c_double), ("storage_precision", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("block_size", ctypes.c_int)]


_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p
_CTX = ctypes.c_void_p

# (name, restype, argtypes) of every entry point in include/hisq.h
_PROTOS = [
    ("hisq_default_solve_params", None, [ctypes.POINTER(hisq_solve_params)]),
    ("hisq_default_eig_params", None, [ctypes.POINTER(hisq_eig_params)]),
    ("hisq_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, _VP,
                                   ctypes.POINTER(_CTX)]),
    ("hisq_destroy", None, [_CTX]),
    ("hisq_last_error", ctypes.c_char_p, [_CTX]),
    ("hisq_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("hisq_load_links", ctypes.c_int, [_CTX, _DP, _DP, ctypes.c_int, ctypes.c_double]),
    ("hisq_set_mass", ctypes.c_int, [_CTX, ctypes.c_double]),
    ("hisq_apply_dslash", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, ctypes.c_int, _DP, _DP]),
    ("hisq_apply_normal_op", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, _DP, _DP]),
    ("hisq_solve", ctypes.c_int, [_CTX, _DP, _DP, ctypes.c_int, ctypes.POINTER(hisq_solve_params),
                                  ctypes.POINTER(hisq_solve_stats)]),
    ("hisq_solve_device", ctypes.c_int, [_CTX, _VP, _VP, ctypes.c_int, ctypes.POINTER(hisq_solve_params),
                                         ctypes.POINTER(hisq_solve_stats)]),
    ("hisq_eigensolve", ctypes.c_int, [_CTX, ctypes.POINTER(hisq_eig_params), ctypes.POINTER(ctypes.c_int), _DP]),
    ("hisq_get_eigvals", ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int), _DP]),
    ("hisq_get_eigvec", ctypes.c_int, [_CTX, ctypes.c_int, _DP]),
    ("hisq_set_eigvecs", ctypes.c_int, [_CTX, ctypes.c_int, _DP, _DP, ctypes.c_int]),
    ("hisq_deflate", ctypes.c_int, [_CTX, ctypes.c_int, _DP, _DP]),
    ("hisq_save_eigvecs", ctypes.c_int, [_CTX, ctypes.c_char_p]),
    ("hisq_load_eigvecs", ctypes.c_int, [_CTX, ctypes.c_char_p]),
    ("hisq_set_profiling", ctypes.c_int, [_CTX, ctypes.c_int]),
    ("hisq_profiled_fp64", ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_ulonglong)]),
    ("hisq_inject_alloc_failure", ctypes.c_int, [_CTX, ctypes.c_int]),
    ("hisq_inject_wait_timeout", ctypes.c_int, [_CTX, ctypes.c_int]),
    ("hisq_set_batched_kernel", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("hisq_apply_dslash_batch", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, ctypes.c_int, _DP, _DP]),
    ("hisq_bounds_violations", ctypes.c_int, [_CTX, ctypes.POINTER(ctypes.c_int)]),
    ("hisq_device_bytes", ctypes.c_size_t, [_CTX]),
    ("hisq_kernel_launches", ctypes.c_ulonglong, [_CTX]),
]


def load_library(path: Optional[str] = None):
    """Load libhisq.so (raises if it is missing: there is no CPU fallback)."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is missing: run paper_2502_00152_gb300.build.build() first")
    lib = ctypes.CDLL(p)
    for name, res, args in _PROTOS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _check(ctx, st: int, allow_not_converged: bool = False) -> int:
    if st == HISQ_OK or (allow_not_converged and st == HISQ_ERR_NOT_CONVERGED):
        return st
    msg = load_library().hisq_last_error(ctx).decode() if ctx else load_library().hisq_status_string(st).decode()
    raise HisqError(st, msg)


def _field(a, V: int, n: int = 1) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128)
    if a.size != n * V * 3:
        raise ValueError(f"field has {a.size} complex entries, expected {n * V * 3}")
    return a


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


# --------------------------------------------------------------- entry points
def hisq_default_solve_params(**kw) -> hisq_solve_params:
    p = hisq_solve_params()
    load_library().hisq_default_solve_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def hisq_default_eig_params(**kw) -> hisq_eig_params:
    p = hisq_eig_params()
    load_library().hisq_default_eig_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Context:
    """Owns one hisq_ctx (destroyed on close / garbage collection)."""

    def __init__(self, handle, dims):
        self.handle = handle
        self.dims = tuple(dims)
        self.V = int(np.prod(dims))

    def close(self):
        if self.handle:
            load_library().hisq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


_CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy


def hisq_create(dims, t_antiperiodic: bool = True, device: int = 0, cuda_stream: Optional[int] = None) -> Context:
    """cuda_stream: a cudaStream_t handle (e.g. torch.cuda.Stream().cuda_stream)
    for the context's work, or None for a stream of the context's own.  Handle 0,
    which is what torch reports for its default stream, means the legacy default
    stream and is passed on as cudaStreamLegacy, so that the library's kernels are
    ordered with torch's work on that stream."""
    lib = load_library()
    d = (ctypes.c_int * 4)(*[int(x) for x in dims])
    h = _CTX()
    if cuda_stream is not None and int(cuda_stream) == 0:
        cuda_stream = _CUDA_STREAM_LEGACY
    st = lib.hisq_create(d, 1 if t_antiperiodic else 0, device, cuda_stream, ctypes.byref(h))
    _check(None, st)
    return Context(h, dims)


def hisq_destroy(ctx: Context) -> None:
    ctx.close()


def hisq_last_error(ctx: Context) -> str:
    return load_library().hisq_last_error(ctx.handle).decode()


def hisq_status_string(status: int) -> str:
    return load_library().hisq_status_string(status).decode()


def hisq_load_links(ctx: Context, fat, lng, long_recon: int = 18, long_scale: float = 1.0) -> None:
    f = np.ascontiguousarray(fat, dtype=np.complex128)
    l = np.ascontiguousarray(lng, dtype=np.complex128)
    if f.size != ctx.V * 36 or l.size != ctx.V * 36:
        raise ValueError("links must have V*4*3*3 complex entries")
    _check(ctx.handle, load_library().hisq_load_links(ctx.handle, _dp(f), _dp(l), long_recon, long_scale))


def hisq_set_mass(ctx: Context, m: float) -> None:
    _check(ctx.handle, load_library().hisq_set_mass(ctx.handle, m))


def _default_link_prec(precision: int, link_precision):
    if link_precision is None:
        return precision if precision in (64, HISQ_PREC_DF64) else 32
    return link_precision


def hisq_apply_dslash(ctx: Context, out_parity: int, precision: int, field, link_precision=None) -> np.ndarray:
    a = _field(field, ctx.V)
    out = np.zeros((ctx.V, 3), dtype=np.complex128)
    lp = _default_link_prec(precision, link_precision)
    _check(ctx.handle, load_library().hisq_apply_dslash(ctx.handle, out_parity, precision, lp, _dp(a), _dp(out)))
    return out


def hisq_apply_normal_op(ctx: Context, precision: int, field, link_precision=None) -> np.ndarray:
    a = _field(field, ctx.V)
    out = np.zeros((ctx.V, 3), dtype=np.complex128)
    lp = _default_link_prec(precision, link_precision)
    _check(ctx.handle, load_library().hisq_apply_normal_op(ctx.handle, precision, lp, _dp(a), _dp(out)))
    return out


def hisq_solve(ctx: Context, eta, params: Optional[hisq_solve_params] = None, guess=None, out=None):
    """Solve M psi = eta for host field(s) eta ((V,3) or (nrhs,V,3)).  With
    params.guess = 1, `guess` (same shape) is the initial guess.  `out`
    (optional, C-contiguous complex128 of eta's shape, e.g. a view of pinned
    host memory) receives psi in place of a newly allocated array.
    Returns (psi, [stats dicts], status)."""
    eta = np.asarray(eta)
    single = eta.ndim == 2
    nrhs = 1 if single else eta.shape[0]
    e = _field(eta, ctx.V, nrhs)
    if out is not None:
        if out.dtype != np.complex128 or not out.flags.c_contiguous or out.size != nrhs * ctx.V * 3:
            raise ValueError("out must be a C-contiguous complex128 array of eta's size")
        psi = out.reshape(nrhs, ctx.V, 3)
    else:
        psi = np.zeros((nrhs, ctx.V, 3), dtype=np.complex128)
    if guess is not None:
        psi[:] = np.asarray(guess, dtype=np.complex128).reshape(psi.shape)
    p = params or hisq_default_solve_params()
    stats = (hisq_solve_stats * max(nrhs, 1))()
    st = load_library().hisq_solve(ctx.handle, _dp(e), _dp(psi), nrhs, ctypes.byref(p), stats)
    _check(ctx.handle, st, allow_not_converged=True)
    out = psi[0] if single else psi
    return out, [stats[i].as_dict() for i in range(nrhs)], st


def hisq_solve_device(ctx: Context, eta_dev, psi_dev, nrhs: int = 1, params: Optional[hisq_solve_params] = None):
    """As hisq_solve on torch CUDA tensors (contiguous, complex128 or float64)."""
    for t in (eta_dev, psi_dev):
        if not t.is_cuda or not t.is_contiguous() or t.element_size() * t.numel() != nrhs * ctx.V * 48:
            raise ValueError("device fields must be contiguous CUDA tensors of nrhs*V*3 complex128")
    p = params or hisq_default_solve_params()
    stats = (hisq_solve_stats * max(nrhs, 1))()
    st = load_library().hisq_solve_device(ctx.handle, ctypes.c_void_p(eta_dev.data_ptr()),
                                          ctypes.c_void_p(psi_dev.data_ptr()), nrhs, ctypes.byref(p), stats)
    _check(ctx.handle, st, allow_not_converged=True)
    return [stats[i].as_dict() for i in range(nrhs)], st


def hisq_eigensolve(ctx: Context, params: hisq_eig_params):
    """Returns (eps ascending, n_conv)."""
    eps = np.zeros(params.n_ev)
    nc = ctypes.c_int(0)
    _check(ctx.handle, load_library().hisq_eigensolve(ctx.handle, ctypes.byref(params), ctypes.byref(nc), _dp(eps)))
    return eps, nc.value


def hisq_get_eigvals(ctx: Context) -> np.ndarray:
    n = ctypes.c_int(0)
    _check(ctx.handle, load_library().hisq_get_eigvals(ctx.handle, ctypes.byref(n), None))
    eps = np.zeros(max(n.value, 1))
    _check(ctx.handle, load_library().hisq_get_eigvals(ctx.handle, ctypes.byref(n), _dp(eps)))
    return eps[: n.value]


def hisq_get_eigvec(ctx: Context, i: int) -> np.ndarray:
    out = np.zeros((ctx.V, 3), dtype=np.complex128)
    _check(ctx.handle, load_library().hisq_get_eigvec(ctx.handle, i, _dp(out)))
    return out


def hisq_set_eigvecs(ctx: Context, vecs, eps=None, storage_precision: int = 32) -> None:
    v = np.asarray(vecs)
    n = v.shape[0]
    v = _field(v, ctx.V, n)
    e = None if eps is None else np.ascontiguousarray(eps, dtype=np.float64)
    _check(ctx.handle, load_library().hisq_set_eigvecs(ctx.handle, n, _dp(v), None if e is None else _dp(e),
                                                       storage_precision))


def hisq_deflate(ctx: Context, b, n: int = 0) -> np.ndarray:
    bb = _field(b, ctx.V)
    out = np.zeros((ctx.V, 3), dtype=np.complex128)
    _check(ctx.handle, load_library().hisq_deflate(ctx.handle, n, _dp(bb), _dp(out)))
    return out


def hisq_save_eigvecs(ctx: Context, path: str) -> None:
    _check(ctx.handle, load_library().hisq_save_eigvecs(ctx.handle, path.encode()))


def hisq_load_eigvecs(ctx: Context, path: str) -> None:
    _check(ctx.handle, load_library().hisq_load_eigvecs(ctx.handle, path.encode()))


def hisq_bounds_violations(ctx: Context) -> int:
    """1 if a kernel of the bounds-checking build met an out-of-range index since
    the last call (raises HisqError with HISQ_ERR_STATE on a normal build)."""
    f = ctypes.c_int(0)
    _check(ctx.handle, load_library().hisq_bounds_violations(ctx.handle, ctypes.byref(f)))
    return f.value


def hisq_inject_alloc_failure(ctx: Context, after: int) -> None:
    """Host-side failure injection: device allocations fail after `after` more
    (after < 0 switches it off)."""
    _check(ctx.handle, load_library().hisq_inject_alloc_failure(ctx.handle, int(after)))


def hisq_set_batched_kernel(ctx: Context, kind: int = 0, rhs_per_thread: int = 0, budget: int = 0) -> None:
    """Launch shape of the batched operator: kind 0 autotuned; 1 register kernel
    with (budget 0) or without (1) the L2 prefetch of the next direction's links;
    2 TMA-fed kernel (budget = blocks per SM, 2..4); 3 packed-pair kernel
    (rhs_per_thread 2 or 4, budget as kind 1)."""
    _check(ctx.handle, load_library().hisq_set_batched_kernel(ctx.handle, kind, rhs_per_thread, budget))


def hisq_apply_dslash_batch(ctx: Context, out_parity: int, precision: int, fields) -> np.ndarray:
    """D on out_parity for host fields (nrhs, V, 3) through the batched operator."""
    f = np.asarray(fields)
    k = f.shape[0]
    a = _field(f, ctx.V, k)
    out = np.zeros((k, ctx.V, 3), dtype=np.complex128)
    _check(ctx.handle, load_library().hisq_apply_dslash_batch(ctx.handle, out_parity, precision, k, _dp(a), _dp(out)))
    return out


def hisq_inject_wait_timeout(ctx: Context, on: bool = True) -> None:
    """Failure injection: the next tensor-core deflation's GEMM issues no copy and
    its bounded waits give up quickly (HISQ_ERR_TIMEOUT); one-shot."""
    _check(ctx.handle, load_library().hisq_inject_wait_timeout(ctx.handle, 1 if on else 0))


def hisq_set_profiling(ctx: Context, on: bool = True) -> None:
    _check(ctx.handle, load_library().hisq_set_profiling(ctx.handle, 1 if on else 0))


def hisq_device_bytes(ctx: Context) -> int:
    return int(load_library().hisq_device_bytes(ctx.handle))


def hisq_profiled_fp64(ctx: Context):
    """(seconds, launches) of the FP64 Dslash launches made while profiling was
    on, CUDA-event timed."""
    sec, n = ctypes.c_double(0), ctypes.c_ulonglong(0)
    _check(ctx.handle, load_library().hisq_profiled_fp64(ctx.handle, ctypes.byref(sec), ctypes.byref(n)))
    return sec.value, int(n.value)


def hisq_kernel_launches(ctx: Context) -> int:
    return int(load_library().hisq_kernel_launches(ctx.handle))


_PROTOS.append(("hisq_deflate_noalloc", ctypes.c_int, [_CTX, ctypes.c_int, _VP, _VP]))


def hisq_deflate_noalloc(ctx: Context, b_dev, x_dev, n: int = 0) -> None:
    """Deflated guess into caller-owned device memory (torch tensors in the
    even-site FP64 layout [colour][Vh] complex); allocates no device memory."""
    for t in (b_dev, x_dev):
        if not t.is_cuda or not t.is_contiguous() or t.element_size() * t.numel() != ctx.V // 2 * 48:
            raise ValueError("fields must be contiguous CUDA tensors of 3*Vh complex128")
    _check(ctx.handle, load_library().hisq_deflate_noalloc(ctx.handle, n, ctypes.c_void_p(b_dev.data_ptr()),
                                                           ctypes.c_void_p(x_dev.data_ptr())))


_PROTOS.append(("hisq_deflate_batch", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, _DP, _DP, _DP]))


def hisq_deflate_batch(ctx: Context, b, n: int = 0):
    """Tensor-core batched deflation of host fields b (nrhs, V, 3): returns
    (x, r) with x_j = V Lambda^-1 V^dag b_j and r_j = b_j - V V^dag b_j."""
    b = np.asarray(b)
    k = b.shape[0]
    bb = _field(b, ctx.V, k)
    x = np.zeros((k, ctx.V, 3), dtype=np.complex128)
    r = np.zeros((k, ctx.V, 3), dtype=np.complex128)
    _check(ctx.handle, load_library().hisq_deflate_batch(ctx.handle, n, k, _dp(bb), _dp(x), _dp(r)))
    return x, r


_PROTOS += [
    ("hisq_net_layer", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, ctypes.c_int, _VP, _VP]),
    ("hisq_net_wgrad", ctypes.c_int, [_CTX, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP]),
    ("hisq_net_adam", ctypes.c_int, [_CTX, ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.c_float, ctypes.c_float,
                                     ctypes.c_float, ctypes.c_float, ctypes.c_int]),
]


def _dev(t):
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def hisq_net_layer(ctx: Context, w, inp, out, w_bf16: bool = False, adjoint: bool = False) -> None:
    """Parallel-transport layer on torch complex64 CUDA tensors: w (Cout, Cin, 9),
    inp (Cin or Cout, V, 3), out (Cout or Cin, V, 3)."""
    cout, cin = int(w.shape[0]), int(w.shape[1])
    _check(ctx.handle, load_library().hisq_net_layer(ctx.handle, cin, cout, _dev(w), 1 if w_bf16 else 0,
                                                     1 if adjoint else 0, _dev(inp), _dev(out)))


def hisq_net_wgrad(ctx: Context, inp, gout, gw) -> None:
    cout, cin = int(gw.shape[0]), int(gw.shape[1])
    _check(ctx.handle, load_library().hisq_net_wgrad(ctx.handle, cin, cout, _dev(inp), _dev(gout), _dev(gw)))


def hisq_net_adam(ctx: Context, w, g, m1, m2, lr: float, step: int, beta1=0.9, beta2=0.999, eps=1e-8) -> None:
    """Adam step in place on float32 views of the tensors (same shapes)."""
    n = int(w.numel() * (2 if w.is_complex() else 1))
    _check(ctx.handle, load_library().hisq_net_adam(ctx.handle, n, _dev(w), _dev(g), _dev(m1), _dev(m2), lr, beta1,
                                                    beta2, eps, step))
