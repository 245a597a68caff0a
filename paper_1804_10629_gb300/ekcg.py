"""Thin Python binding of libekcg (the C ABI declared in include/ekcg.h).

Only argument marshalling lives here: every step of the solve runs in the library's CUDA
kernels.  Device buffers are torch CUDA tensors (torch is used for memory and streams only).
Importing this module does not need a GPU; calling into the library without the built
library raises immediately (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes
import os
import re
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int64, c_longlong, c_void_p
from typing import Optional

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libekcg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "ekcg.h")

EKCG_OK, EKCG_MAXIT, EKCG_EINVAL, EKCG_ENOMEM, EKCG_EBREAKDOWN, EKCG_ETIMEOUT, EKCG_ECUDA = \
    0, 1, -1, -2, -3, -4, -5
VARIANT = {"sre": 0, "sre2": 1, "msdo": 2}
BASIS = {"sstep": 0, "ca5": 1, "ca7": 2, "restructured": 3}
ORTH = {"acholqr": 0, "precholqr": 1}
PRECISION = {"fp64": 0, "fp32_ir": 1}
CONTRACTION = {"fp64": 0, "split": 1}


class ekcg_opts(ctypes.Structure):
    _fields_ = [("variant", c_int), ("basis", c_int), ("orth", c_int), ("precision", c_int),
                ("max_s", c_int), ("max_blocks", c_int), ("max_basis_bytes", c_int64),
                ("breakdown_tol", c_double), ("inner_tol", c_double), ("max_refine", c_int),
                ("profile", c_int), ("contraction", c_int), ("deflate", c_int)]


class EkcgError(RuntimeError):
    def __init__(self, status, where=""):
        self.status = status
        super().__init__(f"{where}: {strerror(status)} ({status}): {last_error()}")


_lib = None


def _declare(L):
    L.ekcg_default_opts.argtypes = [POINTER(ekcg_opts)]
    L.ekcg_default_opts.restype = None
    L.ekcg_setup.argtypes = [c_int64, c_void_p, c_void_p, c_void_p, c_int, c_void_p,
                             POINTER(ekcg_opts), c_void_p, POINTER(c_void_p)]
    L.ekcg_setup.restype = c_int
    solve_args = [c_void_p, c_void_p, c_void_p, c_int, c_double, c_int, c_void_p,
                  POINTER(c_int), c_void_p, c_int, POINTER(c_int)]
    L.ekcg_solve.argtypes = solve_args
    L.ekcg_solve.restype = c_int
    L.ekcg_solve_host.argtypes = solve_args
    L.ekcg_solve_host.restype = c_int
    L.ekcg_destroy.argtypes = [c_void_p]
    L.ekcg_destroy.restype = None
    L.ekcg_strerror.argtypes = [c_int]
    L.ekcg_strerror.restype = c_char_p
    L.ekcg_last_error.argtypes = []
    L.ekcg_last_error.restype = c_char_p
    L.ekcg_shape.argtypes = [c_void_p, POINTER(c_int64), POINTER(c_int), POINTER(c_int64)]
    L.ekcg_shape.restype = c_int
    L.ekcg_get_perm.argtypes = [c_void_p, c_void_p]
    L.ekcg_get_perm.restype = c_int
    L.ekcg_last_stats.argtypes = [c_void_p, POINTER(c_int64), POINTER(c_int64)]
    L.ekcg_last_stats.restype = c_int
    L.ekcg_block_ic0_host.argtypes = [c_int64, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                      c_void_p, c_void_p, c_void_p]
    L.ekcg_block_ic0_host.restype = c_int
    L.ekcg_set_block_jacobi.argtypes = [c_void_p, c_void_p, c_int]
    L.ekcg_set_block_jacobi.restype = c_int
    L.ekcg_wait_selftest.argtypes = [c_longlong, c_void_p]
    L.ekcg_wait_selftest.restype = c_int
    L.ekcg_fp64_fma_rate.argtypes = [c_void_p, POINTER(c_int), POINTER(c_double)]
    L.ekcg_fp64_fma_rate.restype = c_int
    L.ekcg_deflation_stats.argtypes = [c_void_p, POINTER(c_int64)]
    L.ekcg_deflation_stats.restype = c_int
    L.ekcg_set_device_loop.argtypes = [c_void_p, c_int]
    L.ekcg_set_device_loop.restype = c_int
    L.ekcg_device_loop_stats.argtypes = [c_void_p, POINTER(c_int64)]
    L.ekcg_device_loop_stats.restype = c_int
    L.ekcg_set_profile.argtypes = [c_void_p, c_int]
    L.ekcg_set_profile.restype = c_int
    L.ekcg_profile.argtypes = [c_void_p, c_int, POINTER(c_char_p), POINTER(c_double),
                               POINTER(c_int64), POINTER(c_double), POINTER(c_double),
                               POINTER(c_int)]
    L.ekcg_profile.restype = c_int
    L.ekcg_split_T.argtypes = [c_void_p, c_void_p, c_void_p]
    L.ekcg_split_T.restype = c_int
    L.ekcg_gram.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p]
    L.ekcg_gram.restype = c_int
    L.ekcg_gram_noalloc.argtypes = [c_int64, c_void_p, c_int, c_void_p, c_int, c_void_p,
                                    c_void_p]
    L.ekcg_gram_noalloc.restype = c_int
    L.ekcg_sub_xc.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_void_p, c_int,
                              c_void_p, c_int]
    L.ekcg_sub_xc.restype = c_int
    L.ekcg_gram_with.argtypes = [c_void_p, c_void_p, c_int, c_void_p, c_int, c_void_p, c_int]
    L.ekcg_gram_with.restype = c_int
    L.ekcg_spmm.argtypes = [c_void_p, c_void_p, c_void_p, c_int]
    L.ekcg_spmm.restype = c_int
    L.ekcg_permute.argtypes = [c_void_p, c_void_p, c_void_p, c_int]
    L.ekcg_permute.restype = c_int
    L.ekcg_update_values.argtypes = [c_void_p, c_void_p]
    L.ekcg_update_values.restype = c_int
    L.ekcg_grad_A.argtypes = [c_void_p, c_void_p, c_void_p, c_void_p]
    L.ekcg_grad_A.restype = c_int
    L.ekcg_diffusion2d_values.argtypes = [c_void_p, c_int, c_int, c_double, c_double, c_void_p,
                                          c_void_p]
    L.ekcg_diffusion2d_values.restype = c_int
    L.ekcg_diffusion2d_grad_logkappa.argtypes = [c_void_p, c_int, c_int, c_double, c_double,
                                                 c_void_p, c_void_p, c_void_p, c_void_p]
    L.ekcg_diffusion2d_grad_logkappa.restype = c_int
    L.ekcg_batched_setup.argtypes = [c_int, c_void_p, c_void_p, c_void_p, c_void_p, c_int,
                                     c_void_p, POINTER(ekcg_opts), c_void_p, POINTER(c_void_p)]
    L.ekcg_batched_setup.restype = c_int
    L.ekcg_batched_solve.argtypes = [c_void_p, c_void_p, c_int, c_double, c_int, c_void_p,
                                     c_void_p, c_void_p]
    L.ekcg_batched_solve.restype = c_int
    L.ekcg_batched_tune.argtypes = [c_void_p, c_void_p, c_int, c_double, c_int]
    L.ekcg_batched_tune.restype = c_int
    L.ekcg_batched_set_shape.argtypes = [c_void_p, c_int, c_int, c_int]
    L.ekcg_batched_set_shape.restype = c_int
    L.ekcg_batched_info.argtypes = [c_void_p, POINTER(c_int), POINTER(c_int), POINTER(c_int),
                                    POINTER(c_int), POINTER(c_double)]
    L.ekcg_batched_info.restype = c_int
    L.ekcg_batched_precision_switches.argtypes = [c_void_p, POINTER(c_int)]
    L.ekcg_batched_precision_switches.restype = c_int
    L.ekcg_batched_destroy.argtypes = [c_void_p]
    L.ekcg_batched_destroy.restype = None
    L.ekcg_batched_last_error.argtypes = []
    L.ekcg_batched_last_error.restype = c_char_p


def lib():
    """Load libekcg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_1804_10629_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        _declare(L)
        _lib = L
    return _lib


def header_functions():
    """Names of the functions declared in include/ekcg.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ekcg_\w+)\s*\(", txt)))


def strerror(status: int) -> str:
    return lib().ekcg_strerror(status).decode()


def last_error() -> str:
    return lib().ekcg_last_error().decode()


def ekcg_default_opts() -> ekcg_opts:
    o = ekcg_opts()
    lib().ekcg_default_opts(byref(o))
    return o


def _ptr(a) -> int:
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def ekcg_setup(n, rowptr, colind, val, t, part, opts=None, stream=None):
    """Host numpy arrays in; returns an opaque context handle (int)."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    colind = np.ascontiguousarray(colind, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    part = np.ascontiguousarray(part, dtype=np.int32)
    h = c_void_p()
    st = lib().ekcg_setup(int(n), _ptr(rowptr), _ptr(colind), _ptr(val), int(t), _ptr(part),
                          byref(opts) if opts is not None else None,
                          c_void_p(stream) if stream else None, byref(h))
    if st != EKCG_OK:
        raise EkcgError(st, "ekcg_setup")
    return h.value


def ekcg_solve(ctx, b, x0, s, tol, maxit, x, hist_cap=0):
    """Device pointers (torch tensors) b, x0 (or None), x.  Returns (status, iters, hist)."""
    it = c_int(0)
    hl = c_int(0)
    hist = np.zeros(max(hist_cap, 1), dtype=np.float64)
    st = lib().ekcg_solve(ctx, _ptr(b), _ptr(x0) if x0 is not None else None, int(s),
                          float(tol), int(maxit), _ptr(x), byref(it), _ptr(hist),
                          int(hist_cap), byref(hl))
    return st, it.value, hist[:min(hl.value, hist_cap)]


def ekcg_solve_host(ctx, b, x0, s, tol, maxit, x, hist_cap=0):
    """Host numpy arrays b, x0 (or None), x (written).  Returns (status, iters, hist)."""
    it = c_int(0)
    hl = c_int(0)
    hist = np.zeros(max(hist_cap, 1), dtype=np.float64)
    st = lib().ekcg_solve_host(ctx, _ptr(b), _ptr(x0) if x0 is not None else None, int(s),
                               float(tol), int(maxit), _ptr(x), byref(it), _ptr(hist),
                               int(hist_cap), byref(hl))
    return st, it.value, hist[:min(hl.value, hist_cap)]


def ekcg_destroy(ctx):
    if ctx:
        lib().ekcg_destroy(ctx)


def ekcg_shape(ctx):
    n, t, nnz = c_int64(), c_int(), c_int64()
    lib().ekcg_shape(ctx, byref(n), byref(t), byref(nnz))
    return n.value, t.value, nnz.value


def ekcg_get_perm(ctx, n):
    p = np.empty(n, dtype=np.int64)
    st = lib().ekcg_get_perm(ctx, _ptr(p))
    if st != EKCG_OK:
        raise EkcgError(st, "ekcg_get_perm")
    return p


def ekcg_last_stats(ctx):
    kl, sp = c_int64(), c_int64()
    lib().ekcg_last_stats(ctx, byref(kl), byref(sp))
    return kl.value, sp.value


def ekcg_block_ic0_host(A, bpart):
    """(lval, fwd_level, bwd_level) of the host preconditioner setup for a CSR matrix A
    (rows in their given order) and block ids bpart (host computation only)."""
    rp = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.colind, dtype=np.int32)
    va = np.ascontiguousarray(A.val, dtype=np.float64)
    bp = np.ascontiguousarray(bpart, dtype=np.int32)
    lval = np.zeros(len(va))
    fl = np.zeros(A.n, dtype=np.int32)
    bl = np.zeros(A.n, dtype=np.int32)
    st = lib().ekcg_block_ic0_host(A.n, _ptr(rp), _ptr(ci), _ptr(va), _ptr(bp),
                                   int(bp.max()) + 1, _ptr(lval), _ptr(fl), _ptr(bl))
    if st != EKCG_OK:
        raise EkcgError(st, "ekcg_block_ic0_host")
    return lval, fl, bl


def ekcg_wait_selftest(limit_cycles, stream=None):
    """Status of the bounded-wait diagnostic (EKCG_ETIMEOUT when the wait ran out)."""
    return lib().ekcg_wait_selftest(int(limit_cycles), c_void_p(stream))


def ekcg_fp64_fma_rate(stream=None):
    """(SM count, measured float64 FMA rate in TFLOP/s) of the current device."""
    sms, tf = c_int(), c_double()
    _check(lib().ekcg_fp64_fma_rate(c_void_p(stream) if stream else None, byref(sms),
                                    byref(tf)), "ekcg_fp64_fma_rate")
    return sms.value, tf.value


def ekcg_profile(ctx, cap=32):
    """{class: {"ms", "launches", "flops", "bytes"}} of the last solve."""
    names = (c_char_p * cap)()
    ms = (c_double * cap)()
    nl = (c_int64 * cap)()
    fl = (c_double * cap)()
    by = (c_double * cap)()
    cnt = c_int()
    lib().ekcg_profile(ctx, cap, names, ms, nl, fl, by, byref(cnt))
    return {names[i].decode(): {"ms": ms[i], "launches": nl[i], "flops": fl[i], "bytes": by[i]}
            for i in range(min(cnt.value, cap))}


def _check(st, where):
    if st != EKCG_OK:
        raise EkcgError(st, where)


def ekcg_split_T(ctx, r, T):
    _check(lib().ekcg_split_T(ctx, _ptr(r), _ptr(T)), "ekcg_split_T")


def ekcg_gram(ctx, X, p, Y, q, C):
    _check(lib().ekcg_gram(ctx, _ptr(X), int(p), _ptr(Y), int(q), _ptr(C)), "ekcg_gram")


def ekcg_gram_noalloc(n, X, p, Y, q, C, stream=None):
    """C = X^T Y without any device allocation (fixed 2 MiB library scratch); p, q <= 64.
    Enqueued on `stream` (default: torch's current stream); returns without waiting."""
    if not (1 <= p <= 64 and 1 <= q <= 64):
        raise ValueError(f"ekcg_gram_noalloc: p = {p}, q = {q}; the fixed scratch holds one "
                         "64 x 64 tile per CTA, so 1 <= p, q <= 64")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib().ekcg_gram_noalloc(int(n), _ptr(X), int(p), _ptr(Y), int(q), _ptr(C),
                                   c_void_p(stream) if stream else None), "ekcg_gram_noalloc")


def ekcg_sub_xc(ctx, X, p, C, Y, q, OUT, contraction="fp64"):
    """OUT = Y - X C (device tensors, row-major); contraction "fp64" or "split"."""
    _check(lib().ekcg_sub_xc(ctx, _ptr(X), int(p), _ptr(C), _ptr(Y), int(q), _ptr(OUT),
                             CONTRACTION[contraction]), "ekcg_sub_xc")


def ekcg_gram_with(ctx, X, p, Y, q, C, contraction="fp64"):
    """C = X^T Y (device tensors, row-major); contraction "fp64" or "split"."""
    _check(lib().ekcg_gram_with(ctx, _ptr(X), int(p), _ptr(Y), int(q), _ptr(C),
                                CONTRACTION[contraction]), "ekcg_gram_with")


def ekcg_spmm(ctx, W, U, w):
    _check(lib().ekcg_spmm(ctx, _ptr(W), _ptr(U), int(w)), "ekcg_spmm")


def ekcg_permute(ctx, x, y, direction):
    _check(lib().ekcg_permute(ctx, _ptr(x), _ptr(y), int(direction)), "ekcg_permute")


def ekcg_update_values(ctx, val):
    _check(lib().ekcg_update_values(ctx, _ptr(val)), "ekcg_update_values")


def ekcg_grad_A(ctx, lam, x, dval):
    _check(lib().ekcg_grad_A(ctx, _ptr(lam), _ptr(x), _ptr(dval)), "ekcg_grad_A")


def ekcg_diffusion2d_values(ctx, nx, ny, ax, ay, log_kappa, val):
    _check(lib().ekcg_diffusion2d_values(ctx, int(nx), int(ny), float(ax), float(ay),
                                         _ptr(log_kappa), _ptr(val)), "ekcg_diffusion2d_values")


def ekcg_diffusion2d_grad_logkappa(ctx, nx, ny, ax, ay, log_kappa, lam, x, grad):
    _check(lib().ekcg_diffusion2d_grad_logkappa(ctx, int(nx), int(ny), float(ax), float(ay),
                                                _ptr(log_kappa), _ptr(lam), _ptr(x),
                                                _ptr(grad)), "ekcg_diffusion2d_grad_logkappa")


class Solver:
    """Convenience wrapper owning one context (device work on the current torch stream)."""

    def __init__(self, A, t, part, variant="sre", basis="sstep", orth="acholqr",
                 precision="fp64", max_s=8, max_blocks=0, max_basis_bytes=0,
                 breakdown_tol=1e-14, inner_tol=1e-4, max_refine=30, profile=False,
                 stream=None, contraction=None, deflate=False):
        import torch
        o = ekcg_default_opts()
        o.variant, o.basis, o.orth = VARIANT[variant], BASIS[basis], ORTH[orth]
        o.precision = PRECISION[precision]
        o.max_s, o.max_blocks, o.max_basis_bytes = max_s, max_blocks, max_basis_bytes
        o.breakdown_tol, o.inner_tol, o.max_refine = breakdown_tol, inner_tol, max_refine
        o.profile = int(bool(profile))
        if contraction is not None:          # None: the library default (split products)
            o.contraction = CONTRACTION[contraction]
        o.deflate = int(bool(deflate))
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.n = int(A.n)
        self.nnz = int(A.rowptr[-1])
        self.t = int(t)
        self.ctx = ekcg_setup(A.n, A.rowptr, A.colind, A.val, t, part, o, stream)

    def close(self):
        if getattr(self, "ctx", None):
            ekcg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, x0=None, s=2, tol=1e-8, maxit=1000, hist_cap=4096, x=None):
        import torch
        if x is None:
            x = torch.empty_like(b)
        st, it, hist = ekcg_solve(self.ctx, b, x0, s, tol, maxit, x, hist_cap)
        if st < 0 and st not in (EKCG_EBREAKDOWN, EKCG_ENOMEM):
            raise EkcgError(st, "ekcg_solve")
        return x, it, hist, st

    def solve_host(self, b, x0=None, s=2, tol=1e-8, maxit=1000, hist_cap=4096):
        x = np.empty(self.n, dtype=np.float64)
        st, it, hist = ekcg_solve_host(self.ctx, np.ascontiguousarray(b, dtype=np.float64),
                                       None if x0 is None else np.ascontiguousarray(x0),
                                       s, tol, maxit, x, hist_cap)
        if st < 0 and st not in (EKCG_EBREAKDOWN, EKCG_ENOMEM):
            raise EkcgError(st, "ekcg_solve_host")
        return x, it, hist, st

    def perm(self):
        return ekcg_get_perm(self.ctx, self.n)

    def stats(self):
        return ekcg_last_stats(self.ctx)

    def profile(self):
        return ekcg_profile(self.ctx)

    def set_block_jacobi(self, bpart):
        """Block Jacobi IC(0) preconditioner over the blocks of bpart (natural row order);
        None removes it."""
        if bpart is None:
            st = lib().ekcg_set_block_jacobi(self.ctx, None, 0)
        else:
            bp = np.ascontiguousarray(bpart, dtype=np.int32)
            st = lib().ekcg_set_block_jacobi(self.ctx, _ptr(bp), int(bp.max()) + 1)
        if st != EKCG_OK:
            raise EkcgError(st, "ekcg_set_block_jacobi")

    def set_profile(self, on):
        """Per-launch CUDA-event timing of later solves on or off."""
        lib().ekcg_set_profile(self.ctx, int(bool(on)))

    def set_device_loop(self, on):
        """Device-side convergence test (CUDA graph of conditional iterations) on or off."""
        lib().ekcg_set_device_loop(self.ctx, int(bool(on)))

    def device_loop_iters(self):
        """Iterations of the last solve that ran in the device loop."""
        v = c_int64()
        lib().ekcg_device_loop_stats(self.ctx, byref(v))
        return v.value

    def deflated_columns(self):
        """Columns the rank-revealing A-CholQR dropped in the last solve."""
        v = c_int64()
        lib().ekcg_deflation_stats(self.ctx, byref(v))
        return v.value


class BatchedSolver:
    """Many independent systems (a list of workloads.Problem-like objects with .A and .part)
    solved in one persistent launch (ekcg_batched_*)."""

    def __init__(self, problems, t, precision="fp64", max_s=2, breakdown_tol=1e-14,
                 inner_tol=1e-4, max_refine=30, stream=None):
        import torch
        o = ekcg_default_opts()
        o.precision = PRECISION[precision]
        o.max_s, o.breakdown_tol, o.inner_tol, o.max_refine = max_s, breakdown_tol, inner_tol, \
            max_refine
        self.sizes = np.array([p.A.n for p in problems], dtype=np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)])
        rp = np.concatenate([np.asarray(p.A.rowptr, np.int64) for p in problems])
        ci = np.concatenate([np.asarray(p.A.colind, np.int32) for p in problems])
        va = np.concatenate([np.asarray(p.A.val, np.float64) for p in problems])
        pa = np.concatenate([np.asarray(p.part, np.int32) for p in problems])
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        h = c_void_p()
        st = lib().ekcg_batched_setup(len(problems), _ptr(self.sizes), _ptr(rp), _ptr(ci),
                                      _ptr(va), int(t), _ptr(pa), byref(o), c_void_p(stream),
                                      byref(h))
        if st != EKCG_OK:
            raise RuntimeError(f"ekcg_batched_setup: {strerror(st)}: "
                               f"{lib().ekcg_batched_last_error().decode()}")
        self.h = h.value
        self.nsys = len(problems)

    def solve(self, b, s=2, tol=1e-8, maxit=10000, x=None):
        import torch
        if x is None:
            x = torch.empty_like(b)
        it = np.zeros(self.nsys, dtype=np.int32)
        stt = np.zeros(self.nsys, dtype=np.int32)
        st = lib().ekcg_batched_solve(self.h, _ptr(b), int(s), float(tol), int(maxit), _ptr(x),
                                      _ptr(it), _ptr(stt))
        if st != EKCG_OK:
            raise RuntimeError(f"ekcg_batched_solve: {strerror(st)}: "
                               f"{lib().ekcg_batched_last_error().decode()}")
        return x, it, stt

    def tune(self, b, s=2, tol=1e-8, maxit=10000):
        st = lib().ekcg_batched_tune(self.h, _ptr(b), int(s), float(tol), int(maxit))
        if st != EKCG_OK:
            raise RuntimeError(lib().ekcg_batched_last_error().decode())

    def set_shape(self, threads=512, ctas_per_sm=1, cluster=4):
        st = lib().ekcg_batched_set_shape(self.h, int(threads), int(ctas_per_sm), int(cluster))
        if st != EKCG_OK:
            raise RuntimeError(f"ekcg_batched_set_shape: {strerror(st)}: "
                               f"{lib().ekcg_batched_last_error().decode()}")

    def precision_switches(self):
        """Systems of the last mixed solve that continued in float64 after the float32
        refinement stagnated."""
        v = c_int()
        _check(lib().ekcg_batched_precision_switches(self.h, byref(v)),
               "ekcg_batched_precision_switches")
        return v.value

    def info(self):
        th, cp, cl, gr, ms = c_int(), c_int(), c_int(), c_int(), c_double()
        lib().ekcg_batched_info(self.h, byref(th), byref(cp), byref(cl), byref(gr), byref(ms))
        return {"threads": th.value, "ctas_per_sm": cp.value, "cluster": cl.value,
                "groups": gr.value, "last_ms": ms.value}

    def close(self):
        if getattr(self, "h", None):
            lib().ekcg_batched_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
