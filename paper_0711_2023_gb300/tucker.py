"""Thin Python binding of libtucker.so (include/tucker.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Tensors are torch tensors
(device memory and the current CUDA stream come from torch); numpy arrays are accepted for host
inputs.  Nothing is computed in Python: if the CUDA library is missing or no GPU is visible the
calls raise, there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from ctypes import POINTER, Structure, c_char_p, c_double, c_int32, c_int64, c_uint32, c_void_p

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtucker.so")

TUCKER_OK, TUCKER_EINVAL, TUCKER_ENOMEM, TUCKER_ECUDA = 0, -1, -2, -3
TUCKER_EEMPTY, TUCKER_ETIMEOUT, TUCKER_EINTERNAL, TUCKER_ENOTCONV = -4, -5, -6, -7
TUCKER_FP64, TUCKER_MIXED = 0, 1
TUCKER_HOST, TUCKER_DEVICE = 0, 1


class tucker_coo(Structure):
    _fields_ = [("dims", c_int64 * 3), ("nnz", c_int64), ("idx", c_void_p * 3),
                ("val", c_void_p), ("where", c_int32)]


class tucker_opts(Structure):
    _fields_ = [("precision", c_int32), ("tol", c_double), ("max_iter", c_int32),
                ("init", c_void_p * 3), ("init_where", c_int32), ("stream", c_void_p),
                ("flags", c_uint32)]


class tucker_result(Structure):
    _fields_ = [("G", c_void_p), ("U", c_void_p * 3), ("fit_history", c_void_p),
                ("where", c_int32), ("fit", c_double), ("iters", c_int32),
                ("rank_deficient", c_int32)]


class tucker4_coo(Structure):
    _fields_ = [("dims", c_int64 * 4), ("nnz", c_int64), ("idx", c_void_p * 4),
                ("val", c_void_p), ("where", c_int32)]


class tucker4_opts(Structure):
    _fields_ = [("precision", c_int32), ("tol", c_double), ("max_iter", c_int32),
                ("init", c_void_p * 4), ("init_where", c_int32), ("stream", c_void_p),
                ("flags", c_uint32)]


class tucker4_result(Structure):
    _fields_ = [("G", c_void_p), ("U", c_void_p * 4), ("fit_history", c_void_p),
                ("where", c_int32), ("fit", c_double), ("iters", c_int32),
                ("rank_deficient", c_int32)]


class TuckerError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        lib = _lib()
        msg = lib.tucker_strerror(status).decode()
        detail = lib.tucker_last_error_detail().decode()
        super().__init__(f"{what}: {msg} ({status})" + (f" [{detail}]" if detail else ""))


_LIB = None

# name -> (restype, argtypes)
_SIGS = {
    "tucker_tensor_create": (c_int32, [POINTER(tucker_coo), c_void_p, POINTER(c_void_p)]),
    "tucker_tensor_destroy": (c_int32, [c_void_p]),
    "tucker_tensor_info": (c_int32, [c_void_p, POINTER(c_int64), POINTER(c_double)]),
    "tucker_hosvd": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts), POINTER(tucker_result)]),
    "tucker_hooi": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts), POINTER(tucker_result)]),
    "tucker_sp": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts), POINTER(tucker_result)]),
    "tucker_mp": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts), POINTER(tucker_result)]),
    "tucker_hooi_batched": (c_int32, [c_int32, c_void_p, POINTER(c_int32), POINTER(tucker_opts),
                                      POINTER(tucker_result)]),
    "tucker_mp_batched": (c_int32, [c_int32, c_void_p, POINTER(c_int32), POINTER(tucker_opts),
                                    POINTER(tucker_result)]),
    "tucker4_tensor_create": (c_int32, [POINTER(tucker4_coo), c_void_p, POINTER(c_void_p)]),
    "tucker4_tensor_destroy": (c_int32, [c_void_p]),
    "tucker4_tensor_info": (c_int32, [c_void_p, POINTER(c_int64), POINTER(c_double)]),
    "tucker4_hosvd": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker4_opts),
                                POINTER(tucker4_result)]),
    "tucker4_hooi": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker4_opts),
                               POINTER(tucker4_result)]),
    "tucker4_sp": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker4_opts),
                             POINTER(tucker4_result)]),
    "tucker4_mp": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker4_opts),
                             POINTER(tucker4_result)]),
    "tucker4_ttmc": (c_int32, [c_void_p, c_int32, c_void_p, POINTER(c_int32), c_void_p,
                               c_void_p]),
    "tucker_stream_create": (c_int32, [POINTER(tucker_coo), c_int64, c_void_p,
                                       POINTER(c_void_p)]),
    "tucker_stream_destroy": (c_int32, [c_void_p]),
    "tucker_stream_info": (c_int32, [c_void_p, POINTER(c_int64), POINTER(c_double),
                                     POINTER(c_int64)]),
    "tucker_sp_streamed": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts),
                                     POINTER(tucker_result), POINTER(c_double)]),
    "tucker_mp_streamed": (c_int32, [c_void_p, POINTER(c_int32), POINTER(tucker_opts),
                                     POINTER(tucker_result), POINTER(c_double)]),
    "tucker_strerror": (c_char_p, [c_int32]),
    "tucker_last_error_detail": (c_char_p, []),
    "tucker_ordering": (c_int32, [c_void_p, c_int32, c_int32, c_int32, POINTER(c_int64), c_void_p,
                                  c_void_p, c_void_p, c_void_p, c_void_p, c_int32]),
    "tucker_unfolding_gram": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p]),
    "tucker_ttmc": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_int32, c_void_p,
                              c_void_p]),
    "tucker_slice_proj": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_int32, c_void_p,
                                    c_void_p]),
    "tucker_gram": (c_int32, [c_void_p, c_int64, c_void_p, c_int64, c_int32, c_void_p, c_void_p]),
    "tucker_eig_topk": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_void_p, c_void_p,
                                  c_void_p]),
    "tucker_core": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, POINTER(c_int32), c_void_p,
                              POINTER(c_double), c_void_p]),
    "tucker_ttmc_mixed": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p, c_int32,
                                    c_void_p, c_void_p, c_int64, c_void_p, c_void_p]),
    "tucker_slice_proj_mixed": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_int32,
                                          c_void_p, c_void_p, c_int64, c_void_p]),
    "tucker_gram_bf16x3": (c_int32, [c_void_p, c_void_p, c_int64, c_int64, c_void_p, c_void_p,
                                     c_int64, c_int64, c_int32, c_void_p, c_void_p]),
    "tucker_gram_fused": (c_int32, [c_void_p, c_int32, c_int32, c_void_p, c_int32, c_int32,
                                    c_void_p, c_int32, c_void_p, c_void_p]),
    "tucker_gemm": (c_int32, [c_void_p, c_int64, c_void_p, c_int64, c_int32, c_int32, c_int64,
                              c_void_p, c_int64, c_void_p]),
    "tucker_gram_noalloc": (c_int32, [c_void_p, c_int64, c_void_p, c_int64, c_int32, c_void_p,
                                      c_void_p]),
    "tucker_profile_enable": (None, [c_int32]),
    "tucker_profile_query": (c_int32, [c_char_p, POINTER(c_int64), POINTER(c_double),
                                       POINTER(c_double), POINTER(c_double)]),
    "tucker_launch_count": (c_int64, []),
    "tucker_autotune_enable": (None, [c_int32]),
    "tucker_autotune_count": (c_int32, []),
    "tucker_autotune_decision": (c_int32, [c_int32, POINTER(c_int32), POINTER(c_int32),
                                           POINTER(c_int32), POINTER(c_double), POINTER(c_double)]),
}


def _lib():
    """Loads libtucker.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_0711_2023_gb300.build.build() (needs nvcc)")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _LIB = lib
    return _LIB


def _check(status: int, what: str):
    if status != TUCKER_OK:
        raise TuckerError(status, what)


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("the Tucker library runs on a CUDA GPU; none is visible")
    return torch


def _stream():
    return c_void_p(_torch().cuda.current_stream().cuda_stream)


def _dptr(t):
    return c_void_p(t.data_ptr())


def _dev_f64(a):
    """A contiguous float64 CUDA tensor holding `a` (torch or numpy)."""
    torch = _torch()
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
    return a.to(device="cuda", dtype=torch.float64).contiguous()


def _J(J):
    return (c_int32 * 3)(*[int(j) for j in J])


class Tensor:
    """Owning wrapper of a tucker_tensor handle (device copy of a COO tensor)."""

    def __init__(self, handle, dims):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)

    def close(self):
        if self.handle:
            _lib().tucker_tensor_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        return tucker_tensor_info(self)


def tucker_tensor_create(idx, val, dims) -> Tensor:
    """idx: int32 [3, nnz] and val: float64 [nnz], either both CUDA tensors (device path) or
    numpy arrays / CPU tensors (copied from host memory by the library)."""
    torch = _torch()
    lib = _lib()
    coo = tucker_coo()
    for a in range(3):
        coo.dims[a] = int(dims[a])
    keep = []
    if isinstance(idx, torch.Tensor) and idx.is_cuda:
        idx_t = idx.to(torch.int32).contiguous()
        val_t = val.to(torch.float64).contiguous()
        keep += [idx_t, val_t]
        coo.nnz = int(val_t.numel())
        for a in range(3):
            coo.idx[a] = idx_t[a].data_ptr() if coo.nnz else None
        coo.val = val_t.data_ptr() if coo.nnz else None
        coo.where = TUCKER_DEVICE
    else:
        idx_h = np.ascontiguousarray(np.asarray(idx), dtype=np.int32)
        val_h = np.ascontiguousarray(np.asarray(val), dtype=np.float64)
        keep += [idx_h, val_h]
        coo.nnz = int(val_h.shape[0])
        for a in range(3):
            coo.idx[a] = idx_h[a].ctypes.data if coo.nnz else None
        coo.val = val_h.ctypes.data if coo.nnz else None
        coo.where = TUCKER_HOST
    h = c_void_p()
    _check(lib.tucker_tensor_create(ctypes.byref(coo), _stream(), ctypes.byref(h)),
           "tucker_tensor_create")
    return Tensor(h, dims)


def tucker_tensor_destroy(X: Tensor):
    X.close()


def tucker_strerror(status: int) -> str:
    return _lib().tucker_strerror(int(status)).decode()


def tucker_last_error_detail() -> str:
    return _lib().tucker_last_error_detail().decode()


def tucker_tensor_info(X: Tensor):
    nnz, n2 = c_int64(), c_double()
    _check(_lib().tucker_tensor_info(X.handle, ctypes.byref(nnz), ctypes.byref(n2)),
           "tucker_tensor_info")
    return int(nnz.value), float(n2.value)


def _opts(precision, tol, max_iter, init):
    o = tucker_opts()
    o.precision = TUCKER_MIXED if precision in ("mixed", TUCKER_MIXED) else TUCKER_FP64
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.init_where = TUCKER_DEVICE
    o.stream = _stream().value
    o.flags = 0
    keep = []
    if init is not None:
        for a in range(3):
            if init[a] is not None:
                t = _dev_f64(init[a])
                keep.append(t)
                o.init[a] = t.data_ptr()
    return o, keep


def _run(fn_name, X: Tensor, J, precision, tol, max_iter, init, out="device"):
    """Calls one method; results land in device memory (out="device") or in pinned host
    memory (out="host", the library copies them back itself)."""
    torch = _torch()
    o, keep = _opts(precision, tol, max_iter, init)
    if out == "host":
        alloc = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory()  # noqa: E731
        where = TUCKER_HOST
    else:
        alloc = lambda shape: torch.empty(shape, dtype=torch.float64, device="cuda")  # noqa: E731
        where = TUCKER_DEVICE
    G = alloc(tuple(int(j) for j in J))
    U = [alloc((X.dims[a], int(J[a]))) for a in range(3)]
    fh = alloc((max(1, int(max_iter)),))
    r = tucker_result()
    r.G = G.data_ptr()
    for a in range(3):
        r.U[a] = U[a].data_ptr()
    r.fit_history = fh.data_ptr()
    r.where = where
    _check(getattr(_lib(), fn_name)(X.handle, _J(J), ctypes.byref(o), ctypes.byref(r)), fn_name)
    iters = int(r.iters)
    return dict(G=G, U=U, fit=float(r.fit), iters=iters,
                fit_history=fh[:iters].cpu().numpy().tolist(), rank_deficient=int(r.rank_deficient))


def tucker_hosvd(X: Tensor, J, precision="fp64", out="device"):
    return _run("tucker_hosvd", X, J, precision, 0.0, 1, None, out)


def tucker_hooi(X: Tensor, J, tol=1e-4, max_iter=50, precision="fp64", init=None, out="device"):
    return _run("tucker_hooi", X, J, precision, tol, max_iter, init, out)


def tucker_sp(X: Tensor, J, C_raw, tol=1e-4, max_iter=50, precision="fp64", out="device"):
    return _run("tucker_sp", X, J, precision, tol, max_iter, [None, None, C_raw], out)


def tucker_mp(X: Tensor, J, tol=1e-4, max_iter=50, precision="fp64", init=None, out="device"):
    return _run("tucker_mp", X, J, precision, tol, max_iter, init, out)


def _run_batched(fn_name, Xs, Js, precision, tol, max_iter):
    torch = _torch()
    count = len(Xs)
    o, keep = _opts(precision, tol, max_iter, None)
    res = (tucker_result * count)()
    outs = []
    Jflat = (c_int32 * (3 * count))(*[int(j) for J in Js for j in J])
    handles = (c_void_p * count)(*[X.handle for X in Xs])
    for t, (X, J) in enumerate(zip(Xs, Js)):
        G = torch.empty(tuple(int(j) for j in J), dtype=torch.float64, device="cuda")
        U = [torch.empty((X.dims[a], int(J[a])), dtype=torch.float64, device="cuda")
             for a in range(3)]
        fh = torch.empty(max(1, int(max_iter)), dtype=torch.float64, device="cuda")
        res[t].G = G.data_ptr()
        for a in range(3):
            res[t].U[a] = U[a].data_ptr()
        res[t].fit_history = fh.data_ptr()
        res[t].where = TUCKER_DEVICE
        outs.append((G, U, fh))
    _check(getattr(_lib(), fn_name)(count, handles, Jflat, ctypes.byref(o), res), fn_name)
    return [dict(G=G, U=U, fit=float(res[t].fit), iters=int(res[t].iters),
                 fit_history=fh[:int(res[t].iters)].cpu().numpy().tolist(),
                 rank_deficient=int(res[t].rank_deficient))
            for t, (G, U, fh) in enumerate(outs)]


def tucker_hooi_batched(Xs, Js, tol=1e-4, max_iter=50, precision="fp64"):
    """HOOI on a list of tensors (core sizes Js) in one call; a list of per-tensor results."""
    return _run_batched("tucker_hooi_batched", Xs, Js, precision, tol, max_iter)


def tucker_mp_batched(Xs, Js, tol=1e-4, max_iter=50, precision="fp64"):
    return _run_batched("tucker_mp_batched", Xs, Js, precision, tol, max_iter)


# ---- step entry points -------------------------------------------------------------------------

def tucker_ordering(X: Tensor, n, m, o, copy=True):
    """Builds ordering (n, m, o) if needed and copies it to host numpy arrays; with copy=False
    only builds it and returns its fiber count."""
    lib = _lib()
    F = c_int64()
    _check(lib.tucker_ordering(X.handle, n, m, o, ctypes.byref(F), None, None, None, None, None,
                               TUCKER_HOST), "tucker_ordering")
    if not copy:
        return int(F.value)
    nnz, _ = tucker_tensor_info(X)
    F = int(F.value)
    root_ptr = np.zeros(X.dims[n] + 1, dtype=np.int64)
    fiber_idx = np.zeros(max(F, 1), dtype=np.int32)
    fiber_ptr = np.zeros(F + 1, dtype=np.int64)
    leaf_idx = np.zeros(max(nnz, 1), dtype=np.int32)
    val = np.zeros(max(nnz, 1), dtype=np.float64)
    _check(lib.tucker_ordering(X.handle, n, m, o, None, root_ptr.ctypes.data,
                               fiber_idx.ctypes.data, fiber_ptr.ctypes.data, leaf_idx.ctypes.data,
                               val.ctypes.data, TUCKER_HOST), "tucker_ordering")
    return dict(root_ptr=root_ptr, fiber_idx=fiber_idx[:F], fiber_ptr=fiber_ptr,
                leaf_idx=leaf_idx[:nnz], val=val[:nnz], nfibers=F)


def tucker_unfolding_gram(X: Tensor, n):
    torch = _torch()
    M = torch.empty((X.dims[n], X.dims[n]), dtype=torch.float64, device="cuda")
    _check(_lib().tucker_unfolding_gram(X.handle, n, _dptr(M), _stream()), "tucker_unfolding_gram")
    return M


def _others(n):
    return [a for a in range(3) if a != n]


def tucker_ttmc(X: Tensor, n, Um, Uo):
    torch = _torch()
    m, o = _others(n)
    Um, Uo = _dev_f64(Um), _dev_f64(Uo)
    Y = torch.empty((X.dims[n], Um.shape[1] * Uo.shape[1]), dtype=torch.float64, device="cuda")
    _check(_lib().tucker_ttmc(X.handle, n, _dptr(Um), Um.shape[1], _dptr(Uo), Uo.shape[1],
                              _dptr(Y), _stream()), "tucker_ttmc")
    return Y


def tucker_slice_proj(X: Tensor, n, m, Um):
    torch = _torch()
    o = 3 - n - m
    Um = _dev_f64(Um)
    Y = torch.empty((X.dims[n], X.dims[o] * Um.shape[1]), dtype=torch.float64, device="cuda")
    _check(_lib().tucker_slice_proj(X.handle, n, m, _dptr(Um), Um.shape[1], _dptr(Y), _stream()),
           "tucker_slice_proj")
    return Y


def tucker_gram(Y1, Y2=None):
    torch = _torch()
    Y1 = _dev_f64(Y1)
    rows = Y1.shape[0]
    M = torch.empty((rows, rows), dtype=torch.float64, device="cuda")
    if Y2 is not None:
        Y2 = _dev_f64(Y2)
    _check(_lib().tucker_gram(_dptr(Y1), Y1.shape[1], _dptr(Y2) if Y2 is not None else None,
                              Y2.shape[1] if Y2 is not None else 0, rows, _dptr(M), _stream()),
           "tucker_gram")
    return M


def tucker_gram_fused(X: Tensor, n, m1, U1, m2=None, U2=None):
    """Mixed-form M = Gram((X x_m1 U1^T)_(n)) (+ the term of m2, U2), fused (I_n <= 256)."""
    torch = _torch()
    U1 = _dev_f32(U1)
    U2 = _dev_f32(U2) if U2 is not None else None
    M = torch.empty((X.dims[n], X.dims[n]), dtype=torch.float64, device="cuda")
    _check(_lib().tucker_gram_fused(X.handle, int(n), int(m1), _dptr(U1), U1.shape[1],
                                    -1 if m2 is None else int(m2),
                                    _dptr(U2) if U2 is not None else None,
                                    U2.shape[1] if U2 is not None else 0, _dptr(M), _stream()),
           "tucker_gram_fused")
    return M


def tucker_gemm(A, B):
    """C = A B in FP64 accuracy on the tensor cores (A: m x K, B: K x n)."""
    torch = _torch()
    A, B = _dev_f64(A), _dev_f64(B)
    m, K = A.shape
    n = B.shape[1]
    C = torch.empty((m, n), dtype=torch.float64, device="cuda")
    _check(_lib().tucker_gemm(_dptr(A), max(K, 1), _dptr(B), n, m, n, K, _dptr(C), n, _stream()),
           "tucker_gemm")
    return C


def tucker_gram_noalloc(Y1, Y2=None, M=None):
    """tucker_gram through the allocation-free entry point.  The output M (rows x rows, float64,
    CUDA) may be passed in; the library itself allocates nothing for this call."""
    torch = _torch()
    Y1 = _dev_f64(Y1)
    rows = Y1.shape[0]
    if M is None:
        M = torch.empty((rows, rows), dtype=torch.float64, device="cuda")
    if Y2 is not None:
        Y2 = _dev_f64(Y2)
    _check(_lib().tucker_gram_noalloc(_dptr(Y1), Y1.shape[1],
                                      _dptr(Y2) if Y2 is not None else None,
                                      Y2.shape[1] if Y2 is not None else 0, rows, _dptr(M),
                                      _stream()), "tucker_gram_noalloc")
    return M


def tucker_eig_topk(M, J, U0=None):
    torch = _torch()
    M = _dev_f64(M)
    n = M.shape[0]
    U = torch.empty((n, int(J)), dtype=torch.float64, device="cuda")
    lam = torch.empty(int(J), dtype=torch.float64, device="cuda")
    U0p = None
    if U0 is not None:
        U0 = _dev_f64(U0)
        U0p = _dptr(U0)
    _check(_lib().tucker_eig_topk(_dptr(M), n, int(J), U0p, _dptr(U), _dptr(lam), _stream()),
           "tucker_eig_topk")
    return U, lam


def tucker_core(X: Tensor, A, B, C):
    torch = _torch()
    A, B, C = _dev_f64(A), _dev_f64(B), _dev_f64(C)
    J = (A.shape[1], B.shape[1], C.shape[1])
    G = torch.empty(J, dtype=torch.float64, device="cuda")
    g2 = c_double()
    _check(_lib().tucker_core(X.handle, _dptr(A), _dptr(B), _dptr(C), _J(J), _dptr(G),
                              ctypes.byref(g2), _stream()), "tucker_core")
    return G, float(g2.value)


def gram_ld(K: int) -> int:
    """Row stride (elements) of a split BF16 matrix with K columns: K rounded up to 64."""
    return (int(K) + 63) // 64 * 64


def _split_buffers(rows, K):
    torch = _torch()
    ld = gram_ld(K)
    hi = torch.empty((rows, ld), dtype=torch.bfloat16, device="cuda")
    lo = torch.empty((rows, ld), dtype=torch.bfloat16, device="cuda")
    return hi, lo, ld


def _dev_f32(a):
    torch = _torch()
    if isinstance(a, np.ndarray):
        a = torch.from_numpy(np.ascontiguousarray(a))
    return a.to(device="cuda", dtype=torch.float32).contiguous()


def tucker_ttmc_mixed(X: Tensor, n, Um, Uo, split=True, fp32=False):
    """Returns (hi, lo, Y32): the split BF16 Y_(n) (rows padded to 64 columns) and/or FP32 Y_(n)."""
    torch = _torch()
    Um, Uo = _dev_f32(Um), _dev_f32(Uo)
    K = Um.shape[1] * Uo.shape[1]
    hi = lo = Y32 = None
    ld = 0
    if split:
        hi, lo, ld = _split_buffers(X.dims[n], K)
    if fp32:
        Y32 = torch.empty((X.dims[n], K), dtype=torch.float32, device="cuda")
    _check(_lib().tucker_ttmc_mixed(X.handle, n, _dptr(Um), Um.shape[1], _dptr(Uo), Uo.shape[1],
                                    _dptr(hi) if split else None, _dptr(lo) if split else None,
                                    ld, _dptr(Y32) if fp32 else None, _stream()),
           "tucker_ttmc_mixed")
    return hi, lo, Y32


def tucker_slice_proj_mixed(X: Tensor, n, m, Um):
    o = 3 - n - m
    Um = _dev_f32(Um)
    hi, lo, ld = _split_buffers(X.dims[n], X.dims[o] * Um.shape[1])
    _check(_lib().tucker_slice_proj_mixed(X.handle, n, m, _dptr(Um), Um.shape[1], _dptr(hi),
                                          _dptr(lo), ld, _stream()), "tucker_slice_proj_mixed")
    return hi, lo


def tucker_gram_bf16x3(Y1, Y2=None, K1=None, K2=None):
    """Y1, Y2: (hi, lo) pairs of BF16 CUDA tensors [rows, ld]; K: used columns (default ld)."""
    torch = _torch()
    h1, l1 = Y1
    rows, ld1 = h1.shape
    M = torch.empty((rows, rows), dtype=torch.float64, device="cuda")
    args = [_dptr(h1), _dptr(l1), int(K1 if K1 is not None else ld1), ld1]
    if Y2 is not None:
        h2, l2 = Y2
        args += [_dptr(h2), _dptr(l2), int(K2 if K2 is not None else h2.shape[1]), h2.shape[1]]
    else:
        args += [None, None, 0, 0]
    _check(_lib().tucker_gram_bf16x3(*args, rows, _dptr(M), _stream()), "tucker_gram_bf16x3")
    return M


def tucker_profile_enable(on: bool):
    _lib().tucker_profile_enable(1 if on else 0)


def tucker_profile_query(name: str):
    """(launches, total_ms, algorithmic_flops, algorithmic_bytes) recorded for kernel `name`."""
    n, ms, f, b = c_int64(), c_double(), c_double(), c_double()
    _check(_lib().tucker_profile_query(name.encode(), ctypes.byref(n), ctypes.byref(ms),
                                       ctypes.byref(f), ctypes.byref(b)), "tucker_profile_query")
    return int(n.value), float(ms.value), float(f.value), float(b.value)


def tucker_launch_count() -> int:
    return int(_lib().tucker_launch_count())


def tucker_autotune_enable(on: bool):
    _lib().tucker_autotune_enable(1 if on else 0)


def tucker_autotune_count() -> int:
    return int(_lib().tucker_autotune_count())


def tucker_autotune_decision(i: int):
    """Decision i of the kernel-variant autotuner: dict(family, key, variant, ms_kept, ms_other)."""
    fam, var = c_int32(), c_int32()
    key = (c_int32 * 3)()
    a, b = c_double(), c_double()
    _check(_lib().tucker_autotune_decision(int(i), ctypes.byref(fam), key, ctypes.byref(var),
                                           ctypes.byref(a), ctypes.byref(b)),
           "tucker_autotune_decision")
    return dict(family=int(fam.value), key=tuple(int(k) for k in key), variant=int(var.value),
                ms_kept=float(a.value), ms_other=float(b.value))


def header_functions(header_path=None):
    """Names of the functions declared in include/tucker.h (for export checks)."""
    import re
    path = header_path or os.path.join(os.path.dirname(HERE), "include", "tucker.h")
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tucker_[a-z0-9_]+)\s*\(", text)))


# ---- fourth-order tensors ----------------------------------------------------------------------

class Tensor4(Tensor):
    """Owning wrapper of a tucker4_tensor handle."""

    def close(self):
        if self.handle:
            _lib().tucker4_tensor_destroy(self.handle)
            self.handle = None


def tucker4_tensor_create(idx, val, dims) -> Tensor4:
    """idx: int32 [4, nnz], val: float64 [nnz]; host (numpy / CPU) or CUDA tensors."""
    torch = _torch()
    coo = tucker4_coo()
    for a in range(4):
        coo.dims[a] = int(dims[a])
    if isinstance(idx, torch.Tensor) and idx.is_cuda:
        idx_t = idx.to(torch.int32).contiguous()
        val_t = val.to(torch.float64).contiguous()
        keep = [idx_t, val_t]
        coo.nnz = int(val_t.numel())
        for a in range(4):
            coo.idx[a] = idx_t[a].data_ptr() if coo.nnz else None
        coo.val = val_t.data_ptr() if coo.nnz else None
        coo.where = TUCKER_DEVICE
    else:
        idx_h = np.ascontiguousarray(np.asarray(idx), dtype=np.int32)
        val_h = np.ascontiguousarray(np.asarray(val), dtype=np.float64)
        keep = [idx_h, val_h]
        coo.nnz = int(val_h.shape[0])
        for a in range(4):
            coo.idx[a] = idx_h[a].ctypes.data if coo.nnz else None
        coo.val = val_h.ctypes.data if coo.nnz else None
        coo.where = TUCKER_HOST
    h = c_void_p()
    _check(_lib().tucker4_tensor_create(ctypes.byref(coo), _stream(), ctypes.byref(h)),
           "tucker4_tensor_create")
    del keep
    return Tensor4(h, dims)


def tucker4_tensor_info(X: Tensor4):
    nnz, n2 = c_int64(), c_double()
    _check(_lib().tucker4_tensor_info(X.handle, ctypes.byref(nnz), ctypes.byref(n2)),
           "tucker4_tensor_info")
    return int(nnz.value), float(n2.value)


def _run4(fn_name, X: Tensor4, J, tol, max_iter, init, out="device"):
    torch = _torch()
    o = tucker4_opts()
    o.precision = TUCKER_FP64
    o.tol = float(tol)
    o.max_iter = int(max_iter)
    o.init_where = TUCKER_DEVICE
    o.stream = _stream().value
    o.flags = 0
    keep = []
    if init is not None:
        for a in range(4):
            if init[a] is not None:
                t = _dev_f64(init[a])
                keep.append(t)
                o.init[a] = t.data_ptr()
    if out == "host":
        alloc = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory()  # noqa: E731
        where = TUCKER_HOST
    else:
        alloc = lambda shape: torch.empty(shape, dtype=torch.float64, device="cuda")  # noqa: E731
        where = TUCKER_DEVICE
    G = alloc(tuple(int(j) for j in J))
    U = [alloc((X.dims[a], int(J[a]))) for a in range(4)]
    fh = alloc((max(1, int(max_iter)),))
    r = tucker4_result()
    r.G = G.data_ptr()
    for a in range(4):
        r.U[a] = U[a].data_ptr()
    r.fit_history = fh.data_ptr()
    r.where = where
    Jc = (c_int32 * 4)(*[int(j) for j in J])
    _check(getattr(_lib(), fn_name)(X.handle, Jc, ctypes.byref(o), ctypes.byref(r)), fn_name)
    iters = int(r.iters)
    return dict(G=G, U=U, fit=float(r.fit), iters=iters,
                fit_history=fh[:iters].cpu().numpy().tolist(),
                rank_deficient=int(r.rank_deficient))


def tucker4_hosvd(X: Tensor4, J, out="device"):
    return _run4("tucker4_hosvd", X, J, 0.0, 1, None, out)


def tucker4_hooi(X: Tensor4, J, tol=1e-4, max_iter=50, init=None, out="device"):
    return _run4("tucker4_hooi", X, J, tol, max_iter, init, out)


def tucker4_sp(X: Tensor4, J, D_raw, tol=1e-4, max_iter=50, out="device"):
    return _run4("tucker4_sp", X, J, tol, max_iter, [None, None, None, D_raw], out)


def tucker4_mp(X: Tensor4, J, tol=1e-4, max_iter=50, init=None, out="device"):
    return _run4("tucker4_mp", X, J, tol, max_iter, init, out)


def tucker4_ttmc(X: Tensor4, n, U):
    """Z_(n) of Figure hooin (N = 4) for the factors U (U[n] unused): I_n x prod_{a != n} J_a."""
    torch = _torch()
    Ud = [None if a == n else _dev_f64(U[a]) for a in range(4)]
    J = [1 if a == n else int(Ud[a].shape[1]) for a in range(4)]
    cols = int(np.prod([J[a] for a in range(4) if a != n]))
    Y = torch.empty((X.dims[n], cols), dtype=torch.float64, device="cuda")
    ptrs = (c_void_p * 4)(*[None if a == n else Ud[a].data_ptr() for a in range(4)])
    Jc = (c_int32 * 4)(*J)
    _check(_lib().tucker4_ttmc(X.handle, int(n), ctypes.cast(ptrs, c_void_p), Jc, _dptr(Y),
                               _stream()), "tucker4_ttmc")
    return Y


# ---- tensors streamed from host memory -----------------------------------------------------------

class StreamTensor(Tensor):
    """Owning wrapper of a tucker_stream_tensor handle (orderings in pinned host memory)."""

    def close(self):
        if self.handle:
            _lib().tucker_stream_destroy(self.handle)
            self.handle = None


def tucker_stream_create(idx, val, dims, budget) -> StreamTensor:
    """idx int32 [3, nnz], val float64 [nnz] (host or CUDA); budget: device bytes per chunk."""
    torch = _torch()
    coo = tucker_coo()
    for a in range(3):
        coo.dims[a] = int(dims[a])
    if isinstance(idx, torch.Tensor) and idx.is_cuda:
        idx_t = idx.to(torch.int32).contiguous()
        val_t = val.to(torch.float64).contiguous()
        keep = [idx_t, val_t]
        coo.nnz = int(val_t.numel())
        for a in range(3):
            coo.idx[a] = idx_t[a].data_ptr() if coo.nnz else None
        coo.val = val_t.data_ptr() if coo.nnz else None
        coo.where = TUCKER_DEVICE
    else:
        idx_h = np.ascontiguousarray(np.asarray(idx), dtype=np.int32)
        val_h = np.ascontiguousarray(np.asarray(val), dtype=np.float64)
        keep = [idx_h, val_h]
        coo.nnz = int(val_h.shape[0])
        for a in range(3):
            coo.idx[a] = idx_h[a].ctypes.data if coo.nnz else None
        coo.val = val_h.ctypes.data if coo.nnz else None
        coo.where = TUCKER_HOST
    h = c_void_p()
    _check(_lib().tucker_stream_create(ctypes.byref(coo), int(budget), _stream(), ctypes.byref(h)),
           "tucker_stream_create")
    del keep
    return StreamTensor(h, dims)


def tucker_stream_destroy(X: StreamTensor):
    X.close()


def tucker_stream_info(X: StreamTensor):
    nnz, n2, ch = c_int64(), c_double(), c_int64()
    _check(_lib().tucker_stream_info(X.handle, ctypes.byref(nnz), ctypes.byref(n2),
                                     ctypes.byref(ch)), "tucker_stream_info")
    return int(nnz.value), float(n2.value), int(ch.value)


def _run_streamed(fn_name, X, J, tol, max_iter, init, out="device"):
    torch = _torch()
    o, keep = _opts("fp64", tol, max_iter, init)
    if out == "host":
        alloc = lambda shape: torch.empty(shape, dtype=torch.float64).pin_memory()  # noqa: E731
        where = TUCKER_HOST
    else:
        alloc = lambda shape: torch.empty(shape, dtype=torch.float64, device="cuda")  # noqa: E731
        where = TUCKER_DEVICE
    G = alloc(tuple(int(j) for j in J))
    U = [alloc((X.dims[a], int(J[a]))) for a in range(3)]
    fh = alloc((max(1, int(max_iter)),))
    r = tucker_result()
    r.G = G.data_ptr()
    for a in range(3):
        r.U[a] = U[a].data_ptr()
    r.fit_history = fh.data_ptr()
    r.where = where
    moved = c_double()
    _check(getattr(_lib(), fn_name)(X.handle, _J(J), ctypes.byref(o), ctypes.byref(r),
                                    ctypes.byref(moved)), fn_name)
    iters = int(r.iters)
    return dict(G=G, U=U, fit=float(r.fit), iters=iters,
                fit_history=fh[:iters].cpu().numpy().tolist(),
                rank_deficient=int(r.rank_deficient), bytes_streamed=float(moved.value))


def tucker_sp_streamed(X: StreamTensor, J, C_raw, tol=1e-4, max_iter=50, out="device"):
    return _run_streamed("tucker_sp_streamed", X, J, tol, max_iter, [None, None, C_raw], out)


def tucker_mp_streamed(X: StreamTensor, J, tol=1e-4, max_iter=50, init=None, out="device"):
    return _run_streamed("tucker_mp_streamed", X, J, tol, max_iter, init, out)
